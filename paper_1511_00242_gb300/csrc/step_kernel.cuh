// Fused D2Q9 finite-volume step (DUGKS, Sec 2.2; BKG, Sec 2.3) for sm_103a.
//
// Work decomposition.  A warp owns a strip of consecutive columns and marches
// up through H rows.  With FP32 arithmetic each lane holds two adjacent
// columns as a float pair, whose arithmetic issues as paired (.f32x2)
// instructions: 64 columns, outputs i0 .. i0+59, two halo columns on each
// side of which the inner one is used.  With FP64 each lane holds one
// column: 32 columns, outputs i0 .. i0+29.  Each lane keeps the
// reconstruction variable phi of its columns for rows j-1, j, j+1 in
// registers; values of the neighbouring columns come from warp shuffles.
// Rows arrive through a per-warp ring of tensor copies into shared memory;
// lanes exchange nothing through it, and no block-wide barrier is needed.
// Per row and column:
//   1. load f_tilde of row j+1 (9 coalesced loads), cell stage:
//      rho, u (Eq. macro_var), f_eq (Eq. equilibrium),
//      phi = f_bar^+ (DUGKS, Eq. eq_trans_2) or f_tilde^+ (BKG, Eq. bkg_collision)
//   2. ghost values of phi at non-periodic sides (Sec 2.5)
//   3. the x-face west of the cell: phi(x_b - h xi) by linear
//      reconstruction (Eqs. eq_char / bkg_fb; on a uniform mesh Eq. f_left),
//      split into a left part computed for the column to the left and a
//      right part,
//   4. the y-face north of the cell (the south face is the previous row's
//      north face, kept in registers),
//   5. boundary faces: bounce-back / diffuse wall / inflow (Sec 2.5),
//   6. DUGKS: face moments, f_eq at the face and the back-transform to f,
//   7. update f_tilde^{n+1} = f_tilde^+ - dt/|V| sum (xi . n) A f_face
//      (Eqs. eq_update, lwfv, bkg_fv) and store.
// Every face is computed once.  FP32 arithmetic is on deviations
// delta = f_tilde - c_alpha from a fixed reference c_alpha near w_alpha rho0:
// transforms, reconstruction and the flux difference are affine with weights
// summing to one, so the constant drops out and rounding scales with the
// deviation, not with f_tilde itself.  FP64 works on f_tilde directly.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

// Occupancy target of the step kernel: blocks of 256 threads per SM, which
// caps its registers (1: up to 255, 2: 128).  FP64 (one column per lane) per
// scheme; FP32 arithmetic (two columns per lane) for both schemes.
#ifndef DVBE_DUGKS_MINB
#define DVBE_DUGKS_MINB 2
#endif
#ifndef DVBE_BKG_MINB
#define DVBE_BKG_MINB 1
#endif
#ifndef DVBE_PAIR_MINB
#define DVBE_PAIR_MINB 1
#endif
// Inner-strip row loop: 1 = unrolled by three (phi rows rotate by renaming),
// 0 = rolled with register copies; FP64 per scheme, then FP32 per scheme.
#ifndef DVBE_DUGKS_UNROLL
#define DVBE_DUGKS_UNROLL 0
#endif
#ifndef DVBE_BKG_UNROLL
#define DVBE_BKG_UNROLL 1
#endif
#ifndef DVBE_PAIR_DUGKS_UNROLL
#define DVBE_PAIR_DUGKS_UNROLL 1
#endif
#ifndef DVBE_PAIR_BKG_UNROLL
#define DVBE_PAIR_BKG_UNROLL 1
#endif
// The ring kernel of the two-kernel step: 1 = on the side stream beside the
// inner kernel, 0 = after it on the main stream; DVBE_RING_FIRST 1 launches
// it before the inner kernel.
#ifndef DVBE_RING_CONCURRENT
#define DVBE_RING_CONCURRENT 1
#endif
#ifndef DVBE_RING_FIRST
#define DVBE_RING_FIRST 0
#endif
// Shared-memory stages of each warp's row pipeline (rows j and j+1 are held,
// the others are in flight).
#ifndef DVBE_STAGES
#define DVBE_STAGES 5
#endif

namespace dvbe {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

// Row paths compiled into a kernel (Strip::run).
enum { PATH_BOTH = 0, PATH_INNER = 1, PATH_EDGE = 2 };

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
// Cell-stage equilibrium coefficients whose sums are exact in the compute
// precision.  fl(4/9), fl(1/9) and fl(1/36) share one relative rounding error
// (+7.5e-9 in FP32), so with them the collision would add mass and momentum
// at that rate in every cell and step.  Instead
//   mass:      W0 + 4 W1 + 4 W2 = 1 exactly: W2 = 1/36 rounded to a multiple
//              of 2^-26 (FP32) or 2^-55 (FP64), W1 = 4 W2, W0 = 1 - 20 W2;
//   momentum:  2 G1 + 4 G2 = 1 exactly: G2 = 1/12 rounded likewise,
//              G1 = (1 - 4 G2) / 2;
// all representable.  d_eq = W (rho' + rho Q) + G (e . m), with m = sum e d
// and Q = 4.5 (e.U)^2 - 1.5 |U|^2, is Eq. equilibrium regrouped; its mass and
// momentum equal rho' and m up to unbiased rounding of each term.  W and G
// differ from 4/9, 1/9, 1/36, 1/3, 1/12 by less than 1e-7 relative, which
// moves only non-conserved moments (c_s^2 and the third moments) that much.
template <typename Real> struct EqCoef;
template <> struct EqCoef<float> {
  static constexpr float W2 = 1864135.0f / 67108864.0f;     // 2^26
  static constexpr float W1 = 4.0f * W2;
  static constexpr float W0 = 7456541.0f / 16777216.0f;     // 1 - 20 W2, 2^24
  static constexpr float G2 = 5592405.0f / 67108864.0f;     // 2^26
  static constexpr float G1 = 11184811.0f / 33554432.0f;    // (1 - 4 G2) / 2, 2^25
};
template <> struct EqCoef<double> {
  static constexpr double W2 = 1000799917193444.0 / 36028797018963968.0; // 2^55
  static constexpr double W1 = 4.0 * W2;
  static constexpr double W0 = 4003199668773772.0 / 9007199254740992.0;  // 2^53
  static constexpr double G2 = 3002399751580331.0 / 36028797018963968.0; // 2^55
  static constexpr double G1 = 6004799503160661.0 / 18014398509481984.0; // 2^54
};
static_assert(EqCoef<float>::W0 + 4.0f * EqCoef<float>::W1 + 4.0f * EqCoef<float>::W2 == 1.0f, "");
static_assert(2.0f * EqCoef<float>::G1 + 4.0f * EqCoef<float>::G2 == 1.0f, "");
static_assert(EqCoef<double>::W0 + 4.0 * EqCoef<double>::W1 + 4.0 * EqCoef<double>::W2 == 1.0, "");
static_assert(2.0 * EqCoef<double>::G1 + 4.0 * EqCoef<double>::G2 == 1.0, "");
static_assert(EqCoef<float>::W0 == 1.0f - 20.0f * EqCoef<float>::W2, "");
static_assert(EqCoef<double>::W0 == 1.0 - 20.0 * EqCoef<double>::W2, "");
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
// Codec between the stored value x and the value the arithmetic works on:
//   CODEC_ABS     f_tilde itself (reference 0): d = x
//   CODEC_OFFSET  absolute storage, deviation arithmetic: d = x - c, x = c + d
//   CODEC_DEV     deviations stored unscaled: d = x
//   CODEC_SCALED  scaled deviations: d = s x, x = d / s (s a power of two)
enum { CODEC_ABS, CODEC_OFFSET, CODEC_DEV, CODEC_SCALED };
template <> struct StoreT<ST_F64> {
  using T = double;
  using Real = double;
  static constexpr int CODEC = CODEC_ABS;
};
template <> struct StoreT<ST_F32> {
  using T = float;
  using Real = float;
  static constexpr int CODEC = CODEC_OFFSET;
};
template <> struct StoreT<ST_F32_DEV> {
  using T = float;
  using Real = float;
  static constexpr int CODEC = CODEC_DEV;
};
template <> struct StoreT<ST_F16_DEV> {
  using T = __half;
  using Real = float;
  static constexpr int CODEC = CODEC_SCALED;
};
template <> struct StoreT<ST_BF16_DEV> {
  using T = __nv_bfloat16;
  using Real = float;
  static constexpr int CODEC = CODEC_SCALED;
};

__device__ __forceinline__ double to_real(double x) { return x; }
__device__ __forceinline__ float to_real(float x) { return x; }
__device__ __forceinline__ float to_real(__half x) { return __half2float(x); }
__device__ __forceinline__ float to_real(__nv_bfloat16 x) { return __bfloat162float(x); }

// ---- lane vectors -------------------------------------------------------------
// A lane holds the values of NC adjacent columns: V = double (NC = 1) for FP64
// arithmetic, V = F2 (NC = 2) for FP32 arithmetic.  F2 arithmetic uses the
// paired FP32 instructions (add / sub / mul / fma on .f32x2), which do the
// work of both columns in one issue slot; each component is rounded exactly
// as the scalar instruction rounds it.
struct __align__(8) F2 {
  float x, y;
  F2() = default;
  __device__ __forceinline__ F2(float s) : x(s), y(s) {}
  __device__ __forceinline__ F2(float a, float b) : x(a), y(b) {}
};
__device__ __forceinline__ float2 f2v(F2 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ F2 v2f(float2 a) { return F2(a.x, a.y); }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return v2f(__fadd2_rn(f2v(a), f2v(b))); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return v2f(__fmul2_rn(f2v(a), f2v(b))); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  F2 r;
  asm("{ .reg .b64 pa, pb, pc;\n"
      "mov.b64 pa, {%2, %3}; mov.b64 pb, {%4, %5};\n"
      "sub.rn.f32x2 pc, pa, pb; mov.b64 {%0, %1}, pc; }"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) {
  return v2f(__ffma2_rn(f2v(a), f2v(b), f2v(c)));
}
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }

// Value of the column to the left / right (one and two columns away) of each
// of this lane's columns; lanes hold consecutive columns in order.
__device__ __forceinline__ double shift_l(double v) { return __shfl_up_sync(kFull, v, 1); }
__device__ __forceinline__ double shift_r(double v) { return __shfl_down_sync(kFull, v, 1); }
__device__ __forceinline__ double shift_l2(double v) { return __shfl_up_sync(kFull, v, 2); }
__device__ __forceinline__ double shift_r2(double v) { return __shfl_down_sync(kFull, v, 2); }
__device__ __forceinline__ F2 shift_l(F2 v) { return F2(__shfl_up_sync(kFull, v.y, 1), v.x); }
__device__ __forceinline__ F2 shift_r(F2 v) { return F2(v.y, __shfl_down_sync(kFull, v.x, 1)); }
__device__ __forceinline__ F2 shift_l2(F2 v) {
  return F2(__shfl_up_sync(kFull, v.x, 1), __shfl_up_sync(kFull, v.y, 1));
}
__device__ __forceinline__ F2 shift_r2(F2 v) {
  return F2(__shfl_down_sync(kFull, v.x, 1), __shfl_down_sync(kFull, v.y, 1));
}

__device__ __forceinline__ double comp(double v, int) { return v; }
__device__ __forceinline__ float comp(F2 v, int c) { return c ? v.y : v.x; }
__device__ __forceinline__ void set_comp(double &v, int, double s) { v = s; }
__device__ __forceinline__ void set_comp(F2 &v, int c, float s) {
  if (c)
    v.y = s;
  else
    v.x = s;
}

template <typename Real> struct LaneT;
template <> struct LaneT<double> {
  using V = double;
  static constexpr int NC = 1;
};
template <> struct LaneT<float> {
  using V = F2;
  static constexpr int NC = 2;
};

__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
// Single precision: the hardware approximation alone, within about one ulp
// of 1/x.  1/rho only scales U = m / rho, which enters the cell stage through
// the second-order term Q alone (mass and momentum come from rho' and m) and
// the face equilibrium through the flux, which stays conservative; an ulp
// there is below the rounding of the FP32 arithmetic around it.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ F2 rcp(F2 x) { return F2(rcp_approx(x.x), rcp_approx(x.y)); }

// Weight class of a direction: 0 rest, 1 axis, 2 diagonal.
__host__ __device__ constexpr int WCLS(int a) { return a == 0 ? 0 : (a <= 4 ? 1 : 2); }

// Per-case constants in compute precision, one copy per lane column.
template <typename V> struct K {
  V rho0;   // reference density: sum of the reference values (0 for CODEC_ABS)
  V c[3];   // reference value per weight class (CODEC_OFFSET)
  V sc[3];  // storage scale per weight class (CODEC_SCALED)
  V isc[3]; // 1 / storage scale
};

// Stored value (converted to compute precision) -> value the arithmetic works
// on (see the CODEC_* list).
template <int ST, typename V> __device__ __forceinline__ V decode(V v, int a, const K<V> &k) {
  if constexpr (StoreT<ST>::CODEC == CODEC_SCALED)
    return v * k.sc[WCLS(a)];
  else if constexpr (StoreT<ST>::CODEC == CODEC_OFFSET)
    return v - k.c[WCLS(a)];
  else
    return v;
}
// ... and back.
template <int ST, typename V> __device__ __forceinline__ V encode(V v, int a, const K<V> &k) {
  if constexpr (StoreT<ST>::CODEC == CODEC_SCALED)
    return v * k.isc[WCLS(a)];
  else if constexpr (StoreT<ST>::CODEC == CODEC_OFFSET)
    return v + k.c[WCLS(a)];
  else
    return v;
}

// delta_eq_alpha = f_eq_alpha - w rref = w (rho' + rho P(e.U)) with rho' =
// rho - rref, P = 3 eU + 4.5 eU^2 - 1.5 |U|^2 and U = u / c (Eq. equilibrium,
// c_s^2 = c^2/3).  rref is rho0 for deviation arithmetic and 0 otherwise.
template <typename Real>
__device__ __forceinline__ Real deq_of(int a, Real rp, Real rho, Real Ux, Real Uy, Real u15) {
  Real eU = Real(EX(a)) * Ux + Real(EY(a)) * Uy;
  Real P = eU * (Real(3) + Real(4.5) * eU) - u15;
  return Real(WGT(a)) * (rp + rho * P);
}

// Moments of a 9-vector of deviations: rho' = sum d, m = sum e d, U = m / rho.
template <typename V>
__device__ __forceinline__ void moments(const V (&d)[9], V rho0, V &rp, V &rho, V &mx, V &my,
                                        V &Ux, V &Uy) {
  rp = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
  mx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
  my = (d[2] - d[4]) + (d[5] - d[8]) + (d[6] - d[7]);
  rho = rho0 + rp;
  const V ri = rcp(rho);
  Ux = mx * ri;
  Uy = my * ri;
}

// Cell-stage equilibrium deviation d_eq = W (rho' + rho Q) + G (e . m) with
// the exact-sum coefficients of EqCoef (Eq. equilibrium; P = 3 e.U + Q and
// rho U = m).  Q is even in e, so one value serves a direction and its
// opposite.
template <typename Real, typename V>
__device__ __forceinline__ void cell_deq(V rp, V rho, V mx, V my, V Ux, V Uy, V (&deq)[9]) {
  using C = EqCoef<Real>;
  const V nu15 = V(Real(-1.5)) * vfma(Ux, Ux, Uy * Uy);
  const V up = Ux + Uy, um = Ux - Uy, h = V(Real(4.5));
  const V Qx = vfma(Ux, h * Ux, nu15), Qy = vfma(Uy, h * Uy, nu15);
  const V Qp = vfma(up, h * up, nu15), Qm = vfma(um, h * um, nu15);
  const V r0 = V(C::W0) * rho, r1 = V(C::W1) * rho, r2 = V(C::W2) * rho;
  const V p0 = V(C::W0) * rp, p1 = V(C::W1) * rp, p2 = V(C::W2) * rp;
  const V gx = V(C::G1) * mx, gy = V(C::G1) * my;
  const V gp = V(C::G2) * (mx + my), gm = V(C::G2) * (mx - my);
  deq[0] = vfma(r0, nu15, p0);
  deq[1] = vfma(r1, Qx, p1 + gx);
  deq[3] = vfma(r1, Qx, p1 - gx);
  deq[2] = vfma(r1, Qy, p1 + gy);
  deq[4] = vfma(r1, Qy, p1 - gy);
  deq[5] = vfma(r2, Qp, p2 + gp); // e = (+1, +1)
  deq[7] = vfma(r2, Qp, p2 - gp); // e = (-1, -1)
  deq[8] = vfma(r2, Qm, p2 + gm); // e = (+1, -1)
  deq[6] = vfma(r2, Qm, p2 - gm); // e = (-1, +1)
}

// Boundary rules compiled into the general path: all kinds, or walls only
// (bounce-back and diffuse; periodic sides need no rule).  A smaller general
// path keeps the boundary strips of wall-bounded meshes in the instruction
// cache.
enum { BCS_ALL = 0, BCS_WALLS = 1 };

// Ghost rule for one ghost cell from the first (p1) and second (p2) inner cell.
template <typename Real, bool XSIDE, int BCS = BCS_ALL>
__device__ __forceinline__ void apply_ghost(const SegParam &sp, Real e, Real rho0,
                                            const Real (&p1)[9], const Real (&p2)[9],
                                            Real (&g)[9]) {
  const int kind = sp.kind;
  if (kind == DVBE_BC_WALL_BOUNCEBACK || kind == DVBE_BC_WALL_DIFFUSE) {
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = p1[a] + e * (p1[a] - p2[a]);
  } else if (BCS == BCS_ALL && kind == DVBE_BC_INFLOW_EQ) {
    Real rho = Real(sp.rho), Ux = Real(sp.ux), Uy = Real(sp.uy);
    Real u15 = Real(1.5) * (Ux * Ux + Uy * Uy);
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = deq_of<Real>(a, rho - rho0, rho, Ux, Uy, u15);
  } else if (BCS == BCS_ALL && kind == DVBE_BC_OUTFLOW_ZG) {
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = p1[a];
  } else if (BCS == BCS_ALL && kind == DVBE_BC_OUTFLOW_NEQ) {
    // the first inner value with its equilibrium part at the segment's
    // density: g = p1 + f_eq(rho_s, U_1) - f_eq(rho_1, U_1)
    //            = p1 + w (rho_s - rho_1) (1 + P(U_1))
    Real rp = 0, mx = 0, my = 0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      rp += p1[a];
      mx += Real(EX(a)) * p1[a];
      my += Real(EY(a)) * p1[a];
    }
    const Real rho1 = rho0 + rp, Ux = mx / rho1, Uy = my / rho1;
    const Real u15 = Real(1.5) * (Ux * Ux + Uy * Uy), dr = Real(sp.rho) - rho1;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const Real eU = Real(EX(a)) * Ux + Real(EY(a)) * Uy;
      const Real P = eU * (Real(3) + Real(4.5) * eU) - u15;
      g[a] = p1[a] + Real(WGT(a)) * dr * (Real(1) + P);
    }
  } else if (BCS == BCS_ALL && kind == DVBE_BC_SYMMETRY) {
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = p1[XSIDE ? MIRX(a) : MIRY(a)];
  }
}

// Boundary face treatment (Sec 2.5) on face values fb (deviations), outward
// normal (nx_o, ny_o) of the fluid.  Only the directions crossing the face
// are read or written.
template <typename Real, int BCS = BCS_ALL>
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
  } else if (BCS == BCS_ALL && kind == DVBE_BC_INFLOW_EQ) {
    // free stream: the distributions entering the domain are f_eq of the
    // free-stream state; those leaving keep their reconstructed values
    Real rho = Real(sp.rho), Ux = Real(sp.ux), Uy = Real(sp.uy);
    Real u15 = Real(1.5) * (Ux * Ux + Uy * Uy);
#pragma unroll
    for (int a = 1; a < 9; ++a)
      if (EX(a) * nxo + EY(a) * nyo < 0) fb[a] = deq_of<Real>(a, rho - rho0, rho, Ux, Uy, u15);
  }
}

// DUGKS: face moments of f_bar, f_eq there and f = p f_bar + q f_eq for the
// directions crossing the face (AXIS 0: x-face, e_x != 0; 1: y-face), in
// increment form f = f_bar + q (f_eq - f_bar) (see stage_row).  For
// e.U = +-s, P = s (4.5 s +- 3) - 1.5 |U|^2.
template <typename Real, int AXIS, typename V>
__device__ __forceinline__ void dugks_face(V (&fb)[9], V rho0, V q) {
  V rp, rho, mx, my, Ux, Uy;
  moments(fb, rho0, rp, rho, mx, my, Ux, Uy);
  const V nu15 = V(Real(-1.5)) * vfma(Ux, Ux, Uy * Uy);
  const V w1 = V(Real(WGT(1))), w2 = V(Real(WGT(5)));
  const V r1 = w1 * rho, p1 = w1 * rp, r2 = w2 * rho, p2 = w2 * rp;
  const V up = Ux + Uy, um = Ux - Uy, h = V(Real(4.5)), t3 = V(Real(3)), m3 = V(Real(-3));
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    if ((AXIS == 0 ? EX(a) : EY(a)) == 0) continue;
    const V s = (a == 1 || a == 3) ? Ux : ((a == 2 || a == 4) ? Uy : ((a == 5 || a == 7) ? up : um));
    const bool pos = a == 1 || a == 2 || a == 5 || a == 8;
    const V P = vfma(s, vfma(h, s, pos ? t3 : m3), nu15);
    const V deq = a <= 4 ? vfma(r1, P, p1) : vfma(r2, P, p2);
    fb[a] = vfma(q, deq - fb[a], fb[a]);
  }
}

// Face values each scheme needs: DUGKS all nine (for the face moments), the
// others only the directions crossing the face.
template <int SCHEME> __host__ __device__ constexpr bool needx(int a) {
  return SCHEME == SC_DUGKS ? true : EX(a) != 0;
}
template <int SCHEME> __host__ __device__ constexpr bool needy(int a) {
  return SCHEME == SC_DUGKS ? true : EY(a) != 0;
}

// ---- TMA / mbarrier primitives (inline PTX) ---------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// 3-d tiled bulk tensor copy global -> shared, completion on an mbarrier.
__device__ __forceinline__ void tma_load3(uint32_t dst, const void *tmap, int x, int y, int z,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
// The row copy of one stage, issued by the lanes with on != 0 (lane 0),
// without a branch: expect_tx on the stage's mbarrier, then the tensor copy.
__device__ __forceinline__ void tma_row_pred(uint32_t on, uint32_t bar, uint32_t bytes, uint32_t dst,
                                             const void *tmap, int x, int y) {
  asm volatile(
      "{ .reg .pred p; setp.ne.u32 p, %0, 0;\n"
      "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%1], %2;\n"
      "@p cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%3], [%4, {%5, %6, %7}], [%1]; }" ::"r"(on),
      "r"(bar), "r"(bytes), "r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(0)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_pred(uint32_t on) {
  asm volatile("{ .reg .pred p; setp.ne.u32 p, %0, 0; @p fence.proxy.async.shared::cta; }" ::"r"(on)
               : "memory");
}

// Non-blocking test of an mbarrier phase.
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Test that may suspend the thread for a hardware-defined time.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
template <typename T> __device__ __forceinline__ T lds(uint32_t addr);
template <> __device__ __forceinline__ double lds<double>(uint32_t a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
template <> __device__ __forceinline__ float lds<float>(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
template <> __device__ __forceinline__ __half lds<__half>(uint32_t a) {
  unsigned short v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
  return __ushort_as_half(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 lds<__nv_bfloat16>(uint32_t a) {
  unsigned short v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
  return __ushort_as_bfloat16(v);
}

// Predicated global stores (no branch around the store).
__device__ __forceinline__ void st_pred(double *p, double v, bool on) {
  asm volatile("{ .reg .pred q; setp.ne.b32 q, %2, 0; @q st.global.f64 [%0], %1; }" ::"l"(p), "d"(v),
               "r"((int)on)
               : "memory");
}
__device__ __forceinline__ void st_pred(float *p, float v, bool on) {
  asm volatile("{ .reg .pred q; setp.ne.b32 q, %2, 0; @q st.global.f32 [%0], %1; }" ::"l"(p), "f"(v),
               "r"((int)on)
               : "memory");
}
__device__ __forceinline__ void st_pred(__half *p, float v, bool on) {
  const unsigned short b = __half_as_ushort(__float2half_rn(v));
  asm volatile("{ .reg .pred q; setp.ne.b32 q, %2, 0; @q st.global.b16 [%0], %1; }" ::"l"(p), "h"(b),
               "r"((int)on)
               : "memory");
}
__device__ __forceinline__ void st_pred(__nv_bfloat16 *p, float v, bool on) {
  const unsigned short b = __bfloat16_as_ushort(__float2bfloat16_rn(v));
  asm volatile("{ .reg .pred q; setp.ne.b32 q, %2, 0; @q st.global.b16 [%0], %1; }" ::"l"(p), "h"(b),
               "r"((int)on)
               : "memory");
}

// One lane's NC adjacent values of a staged row (interior strips, where the
// NC columns are aligned: 8 bytes for FP32 pairs, 4 for 16-bit pairs) ...
__device__ __forceinline__ double ld_lane(uint32_t a, const double *) { return lds<double>(a); }
__device__ __forceinline__ F2 ld_lane(uint32_t a, const float *) {
  float x, y;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(a));
  return F2(x, y);
}
__device__ __forceinline__ F2 ld_lane(uint32_t a, const __half *) {
  unsigned v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
  __half2 h;
  memcpy(&h, &v, 4);
  const float2 f = __half22float2(h);
  return F2(f.x, f.y);
}
__device__ __forceinline__ F2 ld_lane(uint32_t a, const __nv_bfloat16 *) {
  unsigned v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
  __nv_bfloat162 h;
  memcpy(&h, &v, 4);
  const float2 f = __bfloat1622float2(h);
  return F2(f.x, f.y);
}
// ... and the predicated store of them.
__device__ __forceinline__ void st_lane(double *p, double v, bool on) { st_pred(p, v, on); }
__device__ __forceinline__ void st_lane(float *p, F2 v, bool on) {
  asm volatile("{ .reg .pred q; setp.ne.b32 q, %3, 0; @q st.global.v2.f32 [%0], {%1, %2}; }" ::"l"(p),
               "f"(v.x), "f"(v.y), "r"((int)on)
               : "memory");
}
__device__ __forceinline__ void st_lane(__half *p, F2 v, bool on) {
  const __half2 h = __floats2half2_rn(v.x, v.y);
  unsigned b;
  memcpy(&b, &h, 4);
  asm volatile("{ .reg .pred q; setp.ne.b32 q, %2, 0; @q st.global.b32 [%0], %1; }" ::"l"(p), "r"(b),
               "r"((int)on)
               : "memory");
}
__device__ __forceinline__ void st_lane(__nv_bfloat16 *p, F2 v, bool on) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
  unsigned b;
  memcpy(&b, &h, 4);
  asm volatile("{ .reg .pred q; setp.ne.b32 q, %2, 0; @q st.global.b32 [%0], %1; }" ::"l"(p), "r"(b),
               "r"((int)on)
               : "memory");
}

// A row copy still pending after CaseArgs::wait_limit polls, or after
// kWaitCycles SM clock cycles (about a second), is a failure: the warp stops
// fetching, waits (with the same bounds) for the copies it has in flight,
// sets bit 1 of the case flag and leaves; the host reports DVBE_ERR_TIMEOUT.
constexpr uint32_t kDrainPolls = 1u << 22;
constexpr long long kWaitCycles = 1ll << 31;

// Shared-memory geometry of one warp's row pipeline for element size ES and
// NC columns per lane.
template <int ES, int NC> struct Pipe {
  static constexpr int W = stage_cols(ES, NC); // columns per staged row
  static constexpr int WW = 16 / ES;           // columns of the periodic-wrap copies
  static constexpr int NS = DVBE_STAGES;       // stages: rows j, j+1 held, the rest in flight
  static constexpr int MAINB = ((9 * W * ES + 127) / 128) * 128;
  // periodic-wrap copies: a 9 x 16-byte box each (fields packed 16 bytes
  // apart); every tensor-copy destination sits on a 128-byte boundary
  static constexpr int WRAPB = 256;
  static constexpr int STAGEB = MAINB + 2 * WRAPB;
  static constexpr int WARPB = NS * STAGEB + 128; // + NS mbarriers, 128-byte multiple
  // tensor-copy destinations (stage, main box, wrap copies) need 128-byte alignment
  static_assert(MAINB % 128 == 0 && WRAPB % 128 == 0 && STAGEB % 128 == 0 && WARPB % 128 == 0,
                "shared-memory layout must keep tensor-copy destinations 128-byte aligned");
  static_assert(9 * W * ES <= MAINB && 9 * 16 <= WRAPB && NS * 8 <= 128, "buffer sizes");
  // pair loads of a staged row need the field stride to keep their alignment
  static_assert((W * ES) % (NC * ES) == 0, "field stride of a staged row");
};

// ---- the strip ---------------------------------------------------------------

template <int SCHEME, int ST, int BCS = BCS_ALL> struct Strip {
  using S = StoreT<ST>;
  using Real = typename S::Real;
  using T = typename S::T;
  using V = typename LaneT<Real>::V;
  static constexpr int NC = LaneT<Real>::NC;   // columns per lane
  static constexpr int COLS = strip_cols_nc(NC); // output columns per strip
  static constexpr int ES = (int)sizeof(T);
  using P = Pipe<ES, NC>;
  static constexpr bool DUG = SCHEME == SC_DUGKS;
  static constexpr bool FD = SCHEME == SC_BKG_FD;
  static constexpr bool CF = SCHEME == SC_CFREE;

  const CaseArgs &A;
  K<V> k;
  int lane, nx, ny, i0, c0, xs, xwrapW;
  int col[NC];       // this lane's columns c0, c0 + 1, ...
  bool valid[NC];    // column holds a cell or a ghost
  bool outc[NC];     // column is an output of this strip
  bool wrapc[NC];    // column comes from a periodic wrap copy
  uint32_t offc[NC]; // byte offset of each column inside a stage (boundary strips)
  uint32_t lds_off;  // byte offset of the first column (inner strips: one aligned load)
  bool per_x, per_y, touchW, touchE, wrapW, wrapE, out_lane;
  // halo columns (A.hx > 0): this strip writes some of them, and this lane
  // writes the copy of its columns at +nx (columns 0 .. hx-1) or -nx
  // (columns nx-hx .. nx-1); inner strips store a lane's columns whole
  bool hstrip, hlo, hhi;
  int xsp; // staged start in the row copy's coordinates (xs + hx)
  V b_phi;       // phi = d + b_phi (d_eq - d)
  V q_face;      // DUGKS face: f = f_bar + q (f_eq - f_bar)
  // x-face coefficients of this lane's columns: right part of the west face,
  // left part of the east face; tangential / update factors of the column
  // (directions of either sign use them with the operands of the difference
  // they multiply swapped, so no negated copies are held).
  V cR[3], cL[3], tR0, tL0, txc, cxu;
  // BKG-FD stencil factors
  Real kx1, kx2, ky1, ky2, kxy;
  int segS[NC], segN[NC];
  T *fout;
  unsigned pitch, plane; // copies of the layout (the argument block is not re-read per row)
  bool bad;
  // row pipeline of this warp
  uint32_t sbase, bbase, txbytes;
  // Fetches are issued and waited for in order through the NS stages, so
  // every stage in one pass of the ring completes a phase of the same parity:
  // islot / cslot are the stages of the next issue / wait and cpar the parity
  // of the current pass.  These persist across the strips a warp processes.
  int islot, cslot;
  uint32_t cpar;
  int nfetch, nissued, nwaited; // of the current strip
  int Fa;                       // logical row of fetch 0
  // Warp-uniform: a wait ran out.  From then on nothing is issued and
  // nothing advances (cslot / cpar stay at the fetch that ran out, nwaited
  // counts the fetches completed before it), so the copies still in flight
  // are fetches nwaited .. nissued-1 on stages cslot, cslot + 1, ...
  bool timeout;
  unsigned long long wlim; // polls before a pending copy counts as lost

  __device__ __forceinline__ Strip(const CaseArgs &args, int lane_, uint32_t sbase_)
      : A(args), lane(lane_), sbase(sbase_) {
    bbase = sbase + P::NS * P::STAGEB;
    islot = 0;
    cslot = 0;
    cpar = 0;
    bad = false;
    timeout = false;
    wlim = args.wait_limit;
  }

  __device__ __forceinline__ void init_barriers() {
    if (lane == 0) {
      for (int s = 0; s < P::NS; ++s) mbar_init(bbase + 8 * s, 1);
      fence_mbar_init();
    }
    __syncwarp();
  }

  __device__ __forceinline__ void setup(int sx) {
    nx = A.nx;
    ny = A.ny;
    per_x = A.per_x;
    per_y = A.per_y;
    i0 = sx * COLS;
    // the strip's lanes hold columns i0 - NC .. i0 + COLS + NC - 1: NC halo
    // columns on each side, of which only the one next to the outputs is used
    c0 = i0 - NC + NC * lane;
    touchW = !per_x && i0 == 0;
    touchE = !per_x && i0 + COLS >= nx;
    const int hx = A.hx;
    wrapW = per_x && i0 == 0 && hx == 0;
    wrapE = per_x && i0 + COLS >= nx && hx == 0;
    // inner strips: lanes 1 .. 30 hold outputs only, all of a lane's columns
    // at once (with halo columns the last strip may end inside a warp; nx is
    // then a multiple of NC)
    out_lane = lane >= 1 && lane <= 30 && c0 + NC - 1 < nx;
    hstrip = hx > 0 && (i0 < hx || i0 + COLS > nx - hx);
    hlo = out_lane && c0 < hx;
    hhi = out_lane && c0 >= nx - hx;
    // staged columns: [xs, xs + W) with xs the aligned start at or left of i0 - NC
    const int al = 16 / ES;
    xs = (i0 - NC >= 0) ? ((i0 - NC) / al) * al : -al;
    xsp = xs + hx;
    lds_off = (uint32_t)((c0 - xs) * ES);
    xwrapW = ((nx - 1) / al) * al;
    txbytes = 9u * P::W * ES + (wrapW ? 9u * 16u : 0u) + (wrapE ? 9u * 16u : 0u);
    const Real *xfth = (const Real *)A.xfth, *xfs = (const Real *)A.xfs;
    const Real *xct = (const Real *)A.xct, *xcu = (const Real *)A.xcu;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int i = c0 + c;
      col[c] = i;
      valid[c] = (i >= 0 && i < nx) || (per_x && (i == -1 || i == nx));
      outc[c] = i >= i0 && i < i0 + COLS && i < nx;
      offc[c] = (uint32_t)((i - xs) * ES);
      wrapc[c] = false;
      // periodic wrap columns come from the wrap copies: column nx-1 for the
      // west halo, column 0 for the east halo
      if (wrapW && i == -1) {
        offc[c] = (uint32_t)(P::MAINB + (nx - 1 - xwrapW) * ES);
        wrapc[c] = true;
      }
      if (wrapE && i == nx) {
        offc[c] = (uint32_t)(P::MAINB + P::WRAPB);
        wrapc[c] = true;
      }
      const int ic = min(max(i, -1), nx);
      const Real thW = xfth[ic + 1], sW = xfs[ic + 1], thE = xfth[ic + 2], sE = xfs[ic + 2];
      set_comp(cR[0], c, thW + sW); // e_x = -1
      set_comp(cR[1], c, thW);
      set_comp(cR[2], c, thW - sW);
      set_comp(cL[0], c, (Real(1) - thE) - sE);
      set_comp(cL[1], c, Real(1) - thE);
      set_comp(cL[2], c, (Real(1) - thE) + sE);
      set_comp(tR0, c, thW);
      set_comp(tL0, c, Real(1) - thE);
      set_comp(txc, c, xct[ic + 1]);
      set_comp(cxu, c, xcu[ic + 1]);
      const int icc = min(max(i, 0), nx - 1);
      segS[c] = per_y ? 0 : A.segid[2][icc];
      segN[c] = per_y ? 0 : A.segid[3][icc];
    }
    // reference density of the arithmetic: rho0 for deviation arithmetic, 0 for
    // FP64 on f_tilde itself
    constexpr int CODEC = StoreT<ST>::CODEC;
    k.rho0 = V(CODEC == CODEC_ABS ? Real(0) : Real(A.rho0));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      k.c[c] = V(Real(0));
      k.sc[c] = V(CODEC == CODEC_SCALED ? Real(A.dev_scale[c]) : Real(1));        // a power of two
      k.isc[c] = V(CODEC == CODEC_SCALED ? Real(1.0 / A.dev_scale[c]) : Real(1)); // exact inverse
    }
    if constexpr (CODEC == CODEC_OFFSET) {
      // c = W rho0 (exact-sum weights): exact when rho0 is a power of two;
      // otherwise rho0 is replaced by the sum of the rounded c
      using C = EqCoef<Real>;
      const Real cw[3] = {Real(C::W0 * A.rho0), Real(C::W1 * A.rho0), Real(C::W2 * A.rho0)};
      for (int c = 0; c < 3; ++c) k.c[c] = V(cw[c]);
      k.rho0 = V(Real(double(cw[0]) + 4.0 * double(cw[1]) + 4.0 * double(cw[2])));
    }
    b_phi = V(Real(A.b_phi));
    q_face = V(Real(A.q_face));
    if constexpr (FD) {
      Real nux = Real(A.fd_nux), nuy = Real(A.fd_nuy);
      kx1 = Real(0.5) * nux;
      kx2 = Real(0.5) * nux * nux;
      ky1 = Real(0.5) * nuy;
      ky2 = Real(0.5) * nuy * nuy;
      kxy = Real(0.25) * nux * nuy;
    }
    fout = (T *)A.fout + hx;
    pitch = (unsigned)A.pitch;
    plane = (unsigned)A.plane;
  }

  // ---- row pipeline: fetch number q of this strip is logical row Fa + q
  template <bool INT> __device__ __forceinline__ void issue() {
    if (timeout) return;
    const uint32_t bar = bbase + 8 * islot, dst = sbase + islot * P::STAGEB;
    const int r = wrapr(Fa + nissued); // periodic in y: rows -1 and ny wrap
    tma_row_pred((uint32_t)(lane == 0), bar, txbytes, dst, &A.tm_main, xsp, r);
    if (!INT && (wrapW || wrapE)) {
      if (lane == 0) {
        if (wrapW) tma_load3(dst + P::MAINB, &A.tm_wrap, xwrapW, r, 0, bar);
        if (wrapE) tma_load3(dst + P::MAINB + P::WRAPB, &A.tm_wrap, 0, r, 0, bar);
      }
    }
    islot = islot + 1 == P::NS ? 0 : islot + 1;
    ++nissued;
  }

  // Bounded wait after a failed first test: every lane polls until all see
  // the phase complete, at most wlim times and kWaitCycles cycles; then the
  // wait has run out.
  __device__ __forceinline__ void wait_slow(uint32_t bar, uint32_t par) {
    const long long t0 = clock64();
    for (unsigned long long n = 0; n < wlim; ++n) {
      if (__all_sync(kFull, mbar_try_wait(bar, par))) return;
      if (__any_sync(kFull, clock64() - t0 > kWaitCycles)) break;
    }
    timeout = true;
  }

  // Wait for the next fetch in order; returns its stage address (after a
  // timeout: the stage of the lost fetch, whose contents are not used).
  __device__ __forceinline__ uint32_t wait() {
    const uint32_t st = sbase + cslot * P::STAGEB, bar = bbase + 8 * cslot;
    if (timeout) return st;
    if (wlim == 0 || !__all_sync(kFull, mbar_test_wait(bar, cpar))) {
      wait_slow(bar, cpar); // a budget of zero polls runs out at once
      if (timeout) return st;
    }
    ++nwaited;
    if (++cslot == P::NS) {
      cslot = 0;
      cpar ^= 1u;
    }
    return st;
  }

  // The oldest held stage is no longer read: reuse it for the next fetch.
  template <bool INT> __device__ __forceinline__ void release() {
    if (nissued < nfetch) {
      __syncwarp();
      fence_proxy_async_pred((uint32_t)(lane == 0));
      issue<INT>();
    }
  }

  template <bool INT> __device__ __forceinline__ void read_row(uint32_t stage, V (&d)[9]) {
    if (INT) {
      const uint32_t base = stage + lds_off;
#pragma unroll
      for (int a = 0; a < 9; ++a) d[a] = decode<ST>(ld_lane(base + a * P::W * ES, (const T *)nullptr), a, k);
    } else {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        V v;
#pragma unroll
        for (int c = 0; c < NC; ++c)
          set_comp(v, c, to_real(lds<T>(stage + offc[c] + a * (wrapc[c] ? 16u : (uint32_t)(P::W * ES)))));
        d[a] = decode<ST>(v, a, k);
      }
    }
  }

  // Cell stage of a staged row r, then the x ghosts:
  // phi = d + b (d_eq - d), d_eq from cell_deq (mass and momentum exact up to
  // unbiased rounding).  The increment form keeps a state at equilibrium
  // exactly in place: with rounded coefficients a d + b d_eq would shift it
  // by (a + b - 1) d every step.
  template <bool INT>
  __device__ __forceinline__ void stage_row(int r, uint32_t stage, V (&phi)[9]) {
    V d[9];
    read_row<INT>(stage, d);
    V rp, rho, mx, my, Ux, Uy;
    moments(d, k.rho0, rp, rho, mx, my, Ux, Uy);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const Real rc = comp(rho, c);
      bad |= valid[c] && !(rc > Real(0) && rc < Real(1e30));
    }
    V deq[9];
    cell_deq<Real>(rp, rho, mx, my, Ux, Uy, deq);
#pragma unroll
    for (int a = 0; a < 9; ++a) phi[a] = vfma(b_phi, deq[a] - d[a], d[a]);
    if (!INT && (touchW || touchE)) ghost_x(r, phi);
  }

  // Boundary rules are applied per column on scalar copies.
  __device__ __forceinline__ void get(const V (&v)[9], int c, Real (&s)[9]) const {
#pragma unroll
    for (int a = 0; a < 9; ++a) s[a] = comp(v[a], c);
  }
  __device__ __forceinline__ void put(V (&v)[9], int c, const Real (&s)[9]) const {
#pragma unroll
    for (int a = 0; a < 9; ++a) set_comp(v[a], c, s[a]);
  }

  __device__ __forceinline__ void ghost_x(int r, V (&phi)[9]) {
    V q1[9], q2[9];
    if (touchW) {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        q1[a] = shift_r(phi[a]);
        q2[a] = shift_r2(phi[a]);
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (col[c] == -1) {
          Real s1[9], s2[9], g[9];
          get(q1, c, s1);
          get(q2, c, s2);
          get(phi, c, g);
          apply_ghost<Real, true, BCS>(A.seg[0][A.segid[0][r]], Real(A.ext[0]), comp(k.rho0, 0), s1, s2, g);
          put(phi, c, g);
        }
      }
    }
    if (touchE) {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        q1[a] = shift_l(phi[a]);
        q2[a] = shift_l2(phi[a]);
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (col[c] == nx) {
          Real s1[9], s2[9], g[9];
          get(q1, c, s1);
          get(q2, c, s2);
          get(phi, c, g);
          apply_ghost<Real, true, BCS>(A.seg[1][A.segid[1][r]], Real(A.ext[1]), comp(k.rho0, 0), s1, s2, g);
          put(phi, c, g);
        }
      }
    }
  }

  // Ghost row from the first (p1) and second (p2) inner rows; side 2 = S, 3 = N.
  __device__ __forceinline__ void ghost_row(int side, const V (&p1)[9], const V (&p2)[9], V (&g)[9]) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      Real s1[9], s2[9], gs[9];
      get(p1, c, s1);
      get(p2, c, s2);
      get(g, c, gs);
      const SegParam &sp = A.seg[side][side == 2 ? segS[c] : segN[c]];
      apply_ghost<Real, false, BCS>(sp, Real(A.ext[side]), comp(k.rho0, 0), s1, s2, gs);
      put(g, c, gs);
    }
  }

  // Flux values of the x-face west of each of this lane's columns at row j:
  // f_bar at x_b - h xi by linear reconstruction, left part from the column
  // to the left (Eqs. eq_char / bkg_fb).
  template <bool INT>
  __device__ __forceinline__ void xface(int j, Real tyc, const V (&Pm)[9], const V (&P0)[9],
                                        const V (&Pp)[9], V (&F)[9]) {
    const V tL = V(tyc) * tL0, tR = V(tyc) * tR0;
    const V z = V(Real(0)), mtL = z - tL, mtR = z - tR;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      if (!needx<SCHEME>(a)) {
        F[a] = z;
        continue;
      }
      const V PcL = P0[a] * cL[EX(a) + 1];
      if (EY(a) != 0) {
        // left part P0 cL - e_y tL dy, right part P0 cR - e_y tR dy
        const V dy = Pp[a] - Pm[a];
        const V Lp = vfma(EY(a) > 0 ? mtL : tL, dy, PcL);
        const V in = vfma(EY(a) > 0 ? mtR : tR, dy, shift_l(Lp));
        F[a] = vfma(P0[a], cR[EX(a) + 1], in);
      } else {
        F[a] = vfma(P0[a], cR[EX(a) + 1], shift_l(PcL));
      }
    }
    if (!INT && (touchW || touchE)) { // warp-uniform test first
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (col[c] == 0 || col[c] == nx) {
          const int side = col[c] == 0 ? 0 : 1;
          Real s[9];
          get(F, c, s);
          face_bc<Real, BCS>(A.seg[side][A.segid[side][j]], side == 0 ? -1 : 1, 0, comp(k.rho0, 0), s);
          put(F, c, s);
        }
      }
    }
    if constexpr (DUG) dugks_face<Real, 0>(F, k.rho0, q_face);
  }

  // Flux values of the y-face kf (between rows kf-1 and kf) at this lane's
  // columns; Pl = phi of row kf-1, Pu = phi of row kf.
  template <bool INT>
  __device__ __forceinline__ void yface(int kf, Real th, Real s, const V (&Pl)[9], const V (&Pu)[9],
                                        V (&F)[9]) {
    const Real a0 = Real(1) - th, b0 = th;
    const V va0 = V(a0), vb0 = V(b0), ap = V(a0 + s), bm = V(b0 - s), am = V(a0 - s), bp = V(b0 + s);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      if (!needy<SCHEME>(a)) {
        F[a] = V(Real(0));
        continue;
      }
      V B = V(Real(0)), own;
      if (EY(a) == 0 || EX(a) != 0) B = vfma(va0, Pl[a], vb0 * Pu[a]);
      if (EY(a) == 0)
        own = B;
      else if (EY(a) > 0)
        own = vfma(ap, Pl[a], bm * Pu[a]);
      else
        own = vfma(am, Pl[a], bp * Pu[a]);
      if (EX(a) != 0) {
        const V Br = shift_r(B), Bl = shift_l(B);
        own = vfma(txc, EX(a) > 0 ? Bl - Br : Br - Bl, own);
      }
      F[a] = own;
    }
    if (!INT && !per_y && (kf == 0 || kf == ny)) {
      const int side = kf == 0 ? 2 : 3;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        Real sv[9];
        get(F, c, sv);
        face_bc<Real, BCS>(A.seg[side][side == 2 ? segS[c] : segN[c]], 0, side == 2 ? -1 : 1,
                      comp(k.rho0, 0), sv);
        put(F, c, sv);
      }
    }
    if constexpr (DUG) dugks_face<Real, 1>(F, k.rho0, q_face);
  }

  template <bool INT> __device__ __forceinline__ void store_row(int j, const V (&v)[9]) {
    // element offsets fit in 32 bits: buffers are limited to 2^31 elements
    if (INT) {
      const unsigned off = (unsigned)j * pitch + (unsigned)c0;
#pragma unroll
      for (int a = 0; a < 9; ++a) st_lane(fout + (off + a * plane), encode<ST>(v[a], a, k), out_lane);
      if (hstrip) { // warp-uniform: the strips at the two ends of a halo row
        // copies at c0 + nx (hlo) or c0 - nx (hhi): signed, both inside the row
        const int hoff = hlo ? nx : -nx;
#pragma unroll
        for (int a = 0; a < 9; ++a)
          st_lane(fout + ((long long)(off + a * plane) + hoff), encode<ST>(v[a], a, k), hlo || hhi);
      }
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const unsigned off = (unsigned)j * pitch + (unsigned)min(max(col[c], 0), nx - 1);
#pragma unroll
        for (int a = 0; a < 9; ++a) st_pred(fout + (off + a * plane), comp(encode<ST>(v[a], a, k), c), outc[c]);
        if (hstrip) {
          const bool lo = outc[c] && col[c] < A.hx, hi = outc[c] && col[c] >= nx - A.hx;
          const int hoff = lo ? nx : -nx;
#pragma unroll
          for (int a = 0; a < 9; ++a)
            st_pred(fout + ((long long)(off + a * plane) + hoff), comp(encode<ST>(v[a], a, k), c), lo || hi);
        }
      }
    }
  }

  // Logical row L (-1 .. ny) is stored (periodic wrap) unless it is a ghost row.
  __device__ __forceinline__ bool stored(int L) const { return per_y || (L >= 0 && L < ny); }
  __device__ __forceinline__ int wrapr(int L) const { return L < 0 ? L + ny : (L >= ny ? L - ny : L); }

  // Per-row mesh factors of rows jb .. jb+31, one row per lane, broadcast by
  // shuffles: tangential factor and update factor of row j, theta and slope
  // factor of the y-face j+1.
  struct RowTab {
    Real tyc, cyu, th, s;
    int jb;
  };
  __device__ __forceinline__ void load_rows(RowTab &t, int jb) {
    const int j = min(jb + lane, ny - 1);
    t.tyc = ((const Real *)A.yct)[j + 1];
    t.cyu = ((const Real *)A.ycu)[j + 1];
    t.th = ((const Real *)A.yfth)[j + 2];
    t.s = ((const Real *)A.yfs)[j + 2];
    t.jb = jb;
  }

  // One row of the Lax-Wendroff stencil (Eqs. bkgfd, central_schemes).
  template <bool INT>
  __device__ __forceinline__ void update_fd(int j, const V (&Pm)[9], const V (&P0)[9], const V (&Pp)[9]) {
    V v[9];
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
      V M = V(cc) * P0[a];
      if (ey) M = vfma(V(cym), Pm[a], vfma(V(cyp), Pp[a], M));
      if (ex) {
        // column parts for the neighbours: this column is di = +1 for the
        // left neighbour and di = -1 for the right one
        V forL = V(cxp) * P0[a], forR = V(cxm) * P0[a];
        if (ey) {
          const Real kc = Real(ex * ey) * kxy;
          const V dyv = Pp[a] - Pm[a];
          forL = vfma(V(kc), dyv, forL);
          forR = vfma(V(-kc), dyv, forR);
        }
        M = M + (shift_r(forL) + shift_l(forR));
      }
      v[a] = M;
    }
    store_row<INT>(j, v);
  }

  // One full row j: phi of row j+1 into Pc (unless have_next), the faces and
  // the finite-volume update (Eqs. eq_update, lwfv, bkg_fv), accumulated
  // face by face.  DUGKS needs f_tilde^+ of the cell, recomputed from the
  // staged values d and phi = f_bar^+ as f_tilde^+ = (4 phi - d) / 3 =
  // phi + (phi - d) / 3 (the two transforms of Sec 2.2 combined; the
  // increment form keeps equilibrium exact).  Pa, Pb, Pc = phi of rows j-1,
  // j, j+1; stj / stn = stages holding rows j and j+1 (stj is released at
  // the end of the row).  INT: the strip touches no boundary (all its
  // columns and rows j0-1 .. jend are inner cells), so the ghost, wrap and
  // boundary-face code is compiled out.
  template <bool INT>
  __device__ __forceinline__ void row(int j, int jend, bool have_next, RowTab &rt, V (&Pa)[9],
                                      V (&Pb)[9], V (&Pc)[9], V (&FS)[9], uint32_t &stj,
                                      uint32_t &stn) {
    if (j - rt.jb >= 32) load_rows(rt, j);
    const int q = j - rt.jb;
    const Real tyc = __shfl_sync(kFull, rt.tyc, q), cyu = __shfl_sync(kFull, rt.cyu, q);
    const Real th = __shfl_sync(kFull, rt.th, q), sl = __shfl_sync(kFull, rt.s, q);
    bool last_staged = false;
    if (INT || !have_next) {
      if (INT || stored(j + 1)) {
        stn = wait();
        stage_row<INT>(INT ? j + 1 : wrapr(j + 1), stn, Pc);
        last_staged = j + 1 == jend; // only phi of this row is needed
      } else {
        ghost_row(3, Pb, Pa, Pc);
      }
    }
    if constexpr (FD) {
      update_fd<INT>(j, Pa, Pb, Pc);
    } else {
      V v[9];
      if constexpr (DUG) {
        V d[9];
        read_row<INT>(stj, d);
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = vfma(Pb[a] - d[a], V(Real(1.0 / 3.0)), Pb[a]);
      } else if constexpr (CF) {
        // collision-free faces: phi = f^n = (f_tilde + f_tilde^+) / 2, so
        // f_tilde^+ = phi + (phi - d)
        V d[9];
        read_row<INT>(stj, d);
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = Pb[a] + (Pb[a] - d[a]);
      } else {
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = Pb[a];
      }
      {
        V F[9];
        xface<INT>(j, tyc, Pa, Pb, Pc, F);
#pragma unroll
        for (int a = 0; a < 9; ++a)
          if (EX(a) != 0) {
            const V Fr = shift_r(F[a]);
            v[a] = vfma(cxu, EX(a) > 0 ? F[a] - Fr : Fr - F[a], v[a]);
          }
      }
      {
        V F[9];
        yface<INT>(j + 1, th, sl, Pb, Pc, F);
        const V cy = V(cyu);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
          if (EY(a) != 0) {
            v[a] = vfma(cy, EY(a) > 0 ? FS[a] - F[a] : F[a] - FS[a], v[a]);
            FS[a] = F[a];
          }
        }
      }
      store_row<INT>(j, v);
    }
    // the stage of row j is free; on the strip's last row the stage of row
    // j+1 too (released here rather than right after its cell stage, so that
    // the cell stage, faces and update form one block for the scheduler)
    if (last_staged) release<INT>();
    release<INT>();
    stj = stn;
  }

  template <bool INT> __device__ __forceinline__ void run_t(int j0, int jend) {
    const bool ghost_bottom = !INT && j0 == 0 && !per_y;
    Fa = ghost_bottom ? 0 : j0 - 1;
    const int Fb = (INT || stored(jend)) ? jend : jend - 1;
    nfetch = Fb - Fa + 1;
    nissued = 0;
    nwaited = 0;
    while (nissued < nfetch && nissued < P::NS) issue<INT>();
    RowTab rt;
    load_rows(rt, j0);
    V P0[9], P1[9], P2[9], FS[9];
    uint32_t stj, stn = 0;
    bool have_next = false;
    if (ghost_bottom) {
      stj = wait();
      stage_row<INT>(0, stj, P1);
      stn = wait();
      stage_row<INT>(1, stn, P2);
      ghost_row(2, P1, P2, P0);
      have_next = true;
    } else {
      stage_row<INT>(INT ? j0 - 1 : wrapr(j0 - 1), wait(), P0);
      release<INT>(); // row j0-1 contributes phi only
      stj = wait();
      stage_row<INT>(INT ? j0 : wrapr(j0), stj, P1);
    }
    if constexpr (!FD)
      yface<INT>(j0, ((const Real *)A.yfth)[j0 + 1], ((const Real *)A.yfs)[j0 + 1], P0, P1, FS);
    constexpr bool UNROLL = NC == 1 ? (DUG ? DVBE_DUGKS_UNROLL : DVBE_BKG_UNROLL)
                                    : (DUG ? DVBE_PAIR_DUGKS_UNROLL : DVBE_PAIR_BKG_UNROLL);
    if constexpr (INT && UNROLL) {
      // unrolled by three so that the phi rows rotate by renaming
      int j = j0;
      while (true) {
        if (j >= jend) break;
        row<true>(j, jend, false, rt, P0, P1, P2, FS, stj, stn);
        if (++j >= jend) break;
        row<true>(j, jend, false, rt, P1, P2, P0, FS, stj, stn);
        if (++j >= jend) break;
        row<true>(j, jend, false, rt, P2, P0, P1, FS, stj, stn);
        ++j;
      }
    } else {
      // rolled loop with register copies: the boundary path stays small
      for (int j = j0; j < jend; ++j) {
        row<INT>(j, jend, have_next, rt, P0, P1, P2, FS, stj, stn);
        have_next = false;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
          P0[a] = P1[a];
          P1[a] = P2[a];
        }
      }
    }
  }

  // Column strip sx, rows [j0, jend).  PATHS: PATH_BOTH compiles both row
  // paths and picks the inner one for strips that touch no boundary;
  // PATH_INNER only the inner path (every strip given is inner); PATH_EDGE
  // only the general path, which is correct for any strip.
  template <int PATHS> __device__ __forceinline__ void run(int sx, int j0, int jend) {
    setup(sx);
    if constexpr (PATHS == PATH_INNER) {
      run_t<true>(j0, jend);
    } else if constexpr (PATHS == PATH_EDGE) {
      run_t<false>(j0, jend);
    } else {
      // inner strip: its columns i0 - 1 .. i0 + COLS are cells, and so are the
      // rows j0-1 .. jend, or the mesh is periodic in y (rows wrap)
      const bool cols_inner = A.hx > 0 || (i0 >= 1 && i0 + COLS <= nx - 1);
      const bool inner = cols_inner && (per_y || (j0 >= 1 && jend <= ny - 1));
      if (inner)
        run_t<true>(j0, jend);
      else
        run_t<false>(j0, jend);
    }
  }

  // After a wait ran out: give every copy still in flight a bounded time to
  // land before the warp leaves (its shared memory must stay valid until
  // then).  Fetches nwaited .. nissued-1 are outstanding, in ring order from
  // stage cslot with parity cpar (neither advanced after the timeout).
  __device__ __forceinline__ void drain() {
    if (!timeout) return;
    int s = cslot;
    uint32_t par = cpar;
    for (int q = nwaited; q < nissued; ++q) {
      const long long t0 = clock64();
      for (uint32_t n = 0; n < kDrainPolls; ++n)
        if (__all_sync(kFull, mbar_try_wait(bbase + 8 * s, par)) ||
            __any_sync(kFull, clock64() - t0 > kWaitCycles))
          break;
      if (++s == P::NS) {
        s = 0;
        par ^= 1u;
      }
    }
  }
};

// Blocks of 256 threads per SM the step kernel is compiled for.
template <int SCHEME, int ST> __host__ __device__ constexpr int min_blocks() {
  return LaneT<typename StoreT<ST>::Real>::NC == 2
             ? DVBE_PAIR_MINB
             : (SCHEME == SC_DUGKS ? DVBE_DUGKS_MINB : DVBE_BKG_MINB);
}

// Work items of one step.  PART_ALL: every strip of H rows (one kernel).
// PART_INNER: the inner rectangle of strips (CaseArgs::in_*), H rows each.
// PART_EDGE: the ring of strips around it, in pieces of He rows: a band of
// whole-width rows below the rectangle, the strips left and right of it, and
// a band above it.
enum { PART_ALL = 0, PART_INNER = 1, PART_EDGE = 2 };

template <int PART> __device__ __forceinline__ long long part_items(const CaseArgs &A) {
  if constexpr (PART == PART_INNER)
    return (long long)A.in_nx * A.in_ny;
  else if constexpr (PART == PART_EDGE)
    return A.n_edge;
  else
    return (long long)A.strips_x * A.strips_y;
}

template <int PART>
__device__ __forceinline__ void part_item(const CaseArgs &A, long long it, int &sx, int &j0,
                                          int &jend) {
  if constexpr (PART == PART_INNER) {
    sx = A.in_x0 + (int)(it % A.in_nx);
    j0 = (A.in_y0 + (int)(it / A.in_nx)) * A.H;
    jend = min(j0 + A.H, A.ny);
  } else if constexpr (PART == PART_EDGE) {
    const int k = A.H / A.He; // pieces per strip height
    const long long pieces_y = (A.ny + A.He - 1) / A.He;
    const long long r0 = (long long)A.in_y0 * k;
    const long long r1 = min((long long)(A.in_y0 + A.in_ny) * k, pieces_y);
    const long long nex = A.strips_x - A.in_nx; // ring strips beside the rectangle
    long long q, e = it;
    if (e < r0 * A.strips_x) {
      q = e / A.strips_x;
      sx = (int)(e % A.strips_x);
    } else if ((e -= r0 * A.strips_x) < (r1 - r0) * nex) {
      q = r0 + e / nex;
      const int m = (int)(e % nex);
      sx = m < A.in_x0 ? m : m + A.in_nx;
    } else {
      e -= (r1 - r0) * nex;
      q = r1 + e / A.strips_x;
      sx = (int)(e % A.strips_x);
    }
    j0 = (int)q * A.He;
    jend = min(j0 + A.He, A.ny);
  } else {
    sx = (int)(it % A.strips_x);
    j0 = (int)(it / A.strips_x) * A.H;
    jend = min(j0 + A.H, A.ny);
  }
}

template <int PART> __host__ __device__ constexpr int part_paths() {
  return PART == PART_INNER ? PATH_INNER : (PART == PART_EDGE ? PATH_EDGE : PATH_BOTH);
}

// The strips of one part, each warp taking items gw, gw + nw, ...
template <int SCHEME, int ST, int PART, int BCS = BCS_ALL>
__device__ __forceinline__ void step_part(const CaseArgs &A) {
  extern __shared__ __align__(128) unsigned char smem[];
  using P = typename Strip<SCHEME, ST, BCS>::P;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nitems = part_items<PART>(A);
  Strip<SCHEME, ST, BCS> s(A, lane, smem_u32(smem) + wib * P::WARPB);
  s.init_barriers();
  for (long long it = gw; it < nitems; it += nw) {
    int sx, j0, jend;
    part_item<PART>(A, it, sx, j0, jend);
    s.template run<part_paths<PART>()>(sx, j0, jend);
    if (s.timeout) break; // warp-uniform
  }
  if (s.timeout) {
    s.drain();
    if (lane == 0) atomicOr(A.flag, 2u);
  }
  if (__any_sync(kFull, s.bad) && lane == 0) atomicOr(A.flag, 1u);
}

template <int SCHEME, int ST, int PART>
__global__ void __launch_bounds__(256, min_blocks<SCHEME, ST>())
    k_step(const __grid_constant__ CaseArgs A) {
  step_part<SCHEME, ST, PART>(A);
}

// The inner strips alone: without boundary code the kernel needs fewer
// registers than the general path, so more warps fit on an SM.  Register cap
// per thread: DVBE_PAIR_INNER_MAXREG for paired FP32 strips (168: 12 warps
// per SM), and for FP64 the occupancy target of min_blocks.
#ifndef DVBE_PAIR_INNER_MAXREG
#define DVBE_PAIR_INNER_MAXREG 168
#endif
template <int SCHEME, int ST> __host__ __device__ constexpr int inner_maxreg() {
  return LaneT<typename StoreT<ST>::Real>::NC == 2
             ? DVBE_PAIR_INNER_MAXREG
             : (65536 / (256 * min_blocks<SCHEME, ST>()) > 255 ? 255
                                                               : 65536 / (256 * min_blocks<SCHEME, ST>()));
}
template <int SCHEME, int ST>
__global__ void __maxnreg__((inner_maxreg<SCHEME, ST>())) k_step_inner(const __grid_constant__ CaseArgs A) {
  step_part<SCHEME, ST, PART_INNER>(A);
}
// The ring of boundary strips: the general path alone also fits the cap
// with little spilling, so it too runs at the inner kernel's occupancy.
template <int SCHEME, int ST, int BCS>
__global__ void __maxnreg__((inner_maxreg<SCHEME, ST>())) k_step_edge(const __grid_constant__ CaseArgs A) {
  step_part<SCHEME, ST, PART_EDGE, BCS>(A);
}

// Batched form: warps take strips of all cases from one queue.
template <int SCHEME, int ST>
__global__ void __launch_bounds__(256, 1)
    k_step_batch(const CaseArgs *__restrict__ cases, const long long *__restrict__ prefix,
                 int ncases, long long nitems, unsigned long long *queue) {
  extern __shared__ __align__(128) unsigned char smem[];
  using P = typename Strip<SCHEME, ST>::P;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const uint32_t sb = smem_u32(smem) + wib * P::WARPB;
  int pipe_slot = 0;       // stage of this warp's next fetch
  uint32_t pipe_phase = 0; // parity to wait for on each stage
  {
    Strip<SCHEME, ST> s0(cases[0], lane, sb);
    s0.init_barriers();
  }
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
    Strip<SCHEME, ST> s(A, lane, sb);
    s.islot = pipe_slot;
    s.cslot = pipe_slot;
    s.cpar = pipe_phase;
    int sx, j0, jend;
    part_item<PART_ALL>(A, local, sx, j0, jend);
    s.template run<PATH_BOTH>(sx, j0, jend);
    pipe_slot = s.cslot;
    pipe_phase = s.cpar;
    if (__any_sync(kFull, s.bad) && lane == 0) atomicOr(A.flag, 1u);
    if (s.timeout) { // warp-uniform
      s.drain();
      if (lane == 0) atomicOr(A.flag, 2u);
      break;
    }
  }
}

} // namespace dev

template <int ST> constexpr int warp_smem() {
  return dev::Strip<SC_DUGKS, ST>::P::WARPB;
}

template <typename K> cudaError_t allow_smem(K kern, int bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// One step.  Meshes with inner strips: the inner kernel on the main stream
// and the ring kernel on the side stream, forked from and joined back into
// the main stream, so the two run concurrently (the ring's short pieces fill
// the inner kernel's last wave); both read f_in and write disjoint cells of
// f_out.  Otherwise one kernel over every strip.
template <int SCHEME, int ST>
cudaError_t launch_step_scheme(const CaseArgs &a, int blocks, int wpb, const StepStreams &ss) {
  dim3 block(32 * wpb);
  const int smem = wpb * warp_smem<ST>();
  const long long n_inner = (long long)a.in_nx * a.in_ny;
  cudaError_t e = cudaSuccess;
  if (n_inner == 0) {
    auto kern = dev::k_step<SCHEME, ST, dev::PART_ALL>;
    const long long nitems = (long long)a.strips_x * a.strips_y;
    if (blocks <= 0) blocks = (int)((nitems + wpb - 1) / wpb);
    e = allow_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, block, smem, ss.main>>>(a);
    return cudaGetLastError();
  }
  auto ki = dev::k_step_inner<SCHEME, ST>;
  // a mesh whose non-periodic sides are walls only: the smaller general path
  auto ke = a.walls_only ? dev::k_step_edge<SCHEME, ST, dev::BCS_WALLS> : dev::k_step_edge<SCHEME, ST, dev::BCS_ALL>;
  e = allow_smem(ki, smem);
  if (e == cudaSuccess) e = allow_smem(ke, smem);
  if (e != cudaSuccess) return e;
  const bool ring = a.n_edge > 0;
  const bool fork = ring && DVBE_RING_CONCURRENT;
  const cudaStream_t rs = fork ? ss.side : ss.main;
  const int ring_blocks = (int)((a.n_edge + wpb - 1) / wpb);
  if (fork) {
    e = cudaEventRecord(ss.fork, ss.main);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ss.side, ss.fork, 0);
    if (e != cudaSuccess) return e;
  }
  if (ring && DVBE_RING_FIRST) {
    ke<<<ring_blocks, block, smem, rs>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (blocks <= 0) blocks = (int)((n_inner + wpb - 1) / wpb);
  ki<<<blocks, block, smem, ss.main>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess || !ring) return e;
  if (!DVBE_RING_FIRST) {
    ke<<<ring_blocks, block, smem, rs>>>(a);
    e = cudaGetLastError();
  }
  if (fork && e == cudaSuccess) e = cudaEventRecord(ss.join, ss.side);
  if (fork && e == cudaSuccess) e = cudaStreamWaitEvent(ss.main, ss.join, 0);
  return e;
}

template <int ST>
cudaError_t launch_step_impl(int scheme, const CaseArgs &a, int blocks, int wpb, const StepStreams &ss) {
  switch (scheme) {
    case SC_DUGKS:
      return launch_step_scheme<SC_DUGKS, ST>(a, blocks, wpb, ss);
    case SC_BKG_FV:
      return launch_step_scheme<SC_BKG_FV, ST>(a, blocks, wpb, ss);
    case SC_BKG_FD:
      return launch_step_scheme<SC_BKG_FD, ST>(a, blocks, wpb, ss);
    default:
      return launch_step_scheme<SC_CFREE, ST>(a, blocks, wpb, ss);
  }
}

// Resident blocks per SM of the inner-strip kernel (0 if the query fails).
template <int SCHEME, int ST> int inner_blocks_per_sm_scheme(int wpb) {
  auto kern = dev::k_step_inner<SCHEME, ST>;
  const int smem = wpb * warp_smem<ST>();
  int n = 0;
  if (allow_smem(kern, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 32 * wpb, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <int ST> int inner_blocks_per_sm_impl(int scheme, int wpb) {
  switch (scheme) {
    case SC_DUGKS:
      return inner_blocks_per_sm_scheme<SC_DUGKS, ST>(wpb);
    case SC_BKG_FV:
      return inner_blocks_per_sm_scheme<SC_BKG_FV, ST>(wpb);
    case SC_BKG_FD:
      return inner_blocks_per_sm_scheme<SC_BKG_FD, ST>(wpb);
    default:
      return inner_blocks_per_sm_scheme<SC_CFREE, ST>(wpb);
  }
}

template <int ST>
cudaError_t launch_batch_impl(int scheme, const CaseArgs *d_cases, const long long *d_prefix,
                              int ncases, long long nitems, unsigned long long *d_queue,
                              int blocks, int wpb, cudaStream_t s) {
  dim3 block(32 * wpb);
  const int smem = wpb * warp_smem<ST>();
  auto kern = scheme == SC_DUGKS ? dev::k_step_batch<SC_DUGKS, ST> : dev::k_step_batch<SC_BKG_FV, ST>;
  cudaError_t e = allow_smem(kern, smem);
  if (e != cudaSuccess) return e;
  if (blocks <= 0) {
    // persistent grid: as many blocks as fit on the GPU at once
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block.x, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    blocks = (per_sm > 0 ? per_sm : 1) * sms;
  }
  kern<<<blocks, block, smem, s>>>(d_cases, d_prefix, ncases, nitems, d_queue);
  return cudaGetLastError();
}

} // namespace dvbe
