// Internal declarations shared by the host side of libdvbe and its kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dvbe.h"

namespace dvbe {

// Device storage of f_tilde (matches dvbe_precision).
enum StoreMode { ST_F64 = 0, ST_F32 = 1, ST_F32_DEV = 2, ST_F16_DEV = 3, ST_BF16_DEV = 4 };

// Kernel variants: the DUGKS flux (Sec 2.2), the BKG flux in finite-volume
// form (Eq. bkg_fv with the face values of Eq. f_left generalised to
// stretched meshes), BKG as the Lax-Wendroff stencil (Eq. bkgfd), and the
// collision-free faces of Sec 2.4 (Eqs. cfd1, cfd2: the cell f^n reconstructed
// and used as the flux distribution; central = zero slopes in the tables).
enum Scheme { SC_DUGKS = 0, SC_BKG_FV = 1, SC_BKG_FD = 2, SC_CFREE = 3 };

// Halo columns for meshes periodic in x (CaseArgs::hx); 0 keeps plain rows
// and the wrap copies of the edge strips.
#ifndef DVBE_HALO
#define DVBE_HALO 1
#endif

// Boundary strips of meshes whose non-periodic sides are all walls: 1 = the
// general path compiled with the wall rules alone, 0 = with every rule.
#ifndef DVBE_WALLS_PATH
#define DVBE_WALLS_PATH 1
#endif

// Strip geometry.  A warp's lanes hold lane_cols adjacent columns each (two
// for FP32 arithmetic, which then issues paired FP32 instructions; one for
// FP64); NC halo columns on each side leave strip_cols output columns per
// warp row.  A staged row holds stage_cols columns from a 16-byte aligned
// start at or left of the first lane column (the tensor copy needs x * es to
// be a multiple of 16 bytes).
constexpr int lane_cols(int store) { return store == ST_F64 ? 1 : 2; }
constexpr int strip_cols_nc(int nc) { return 30 * nc; }
constexpr int strip_cols(int store) { return strip_cols_nc(lane_cols(store)); }
constexpr int stage_cols(int es, int nc) {
  return ((32 * nc + 16 / es - 1) + 16 / es - 1) / (16 / es) * (16 / es);
}
static_assert(stage_cols(8, 1) == 34 && stage_cols(4, 1) == 36 && stage_cols(2, 1) == 40 &&
                  stage_cols(4, 2) == 68 && stage_cols(2, 2) == 72,
              "staged row widths");

struct SegParam {
  int kind;   // dvbe_bc_kind
  double rho; // wall: unused; inflow: free-stream density
  double ux;  // wall velocity / free-stream velocity, divided by the lattice speed c
  double uy;
};

// Everything one fused step of one case needs.  Plain data so that it can be
// a __grid_constant__ kernel parameter (single solver) or an element of a
// device array (batched form).
struct CaseArgs {
  // Tensor maps of the input buffer, viewed as [9][ny][pitch]: tm_main with
  // a box of one row of the staged columns x 9 fields, tm_wrap with a
  // 16-byte x 9-field box for periodic wrap columns.
  CUtensorMap tm_main;
  CUtensorMap tm_wrap;
  const void *fin;
  void *fout;
  long long plane; // elements per field
  int pitch;       // elements per row
  // Halo columns of a mesh periodic in x (0: none).  Column i of a row sits
  // at element hx + i of it; elements 0 .. hx-1 hold copies of columns
  // nx-hx .. nx-1 and elements nx+hx .. nx+2hx-1 copies of columns 0 ..
  // hx-1, written by the step with the columns themselves.  The row copies
  // of the step read across the wrap from them, so no strip needs wrap code.
  // fin / fout and the tensor maps address the rows from element 0.
  int hx;
  int nx, ny;
  int per_x, per_y;
  int strips_x, strips_y, H; // strip decomposition: strip_cols columns x H rows per warp
  // Partition of the strips for the two-kernel step: the inner rectangle of
  // strips [in_x0, in_x0 + in_nx) x [in_y0, in_y0 + in_ny) (H rows each, the
  // last possibly fewer) touches no boundary, wrapped column or ghost row
  // (rows wrap by the copy coordinate when the mesh is periodic in y) and
  // runs in a kernel compiled without boundary code; the ring of strips
  // around it runs in a second kernel, cut into pieces of He rows (He divides
  // H) for finer work items.  in_nx * in_ny == 0: one kernel covers every
  // strip.
  int in_x0, in_nx, in_y0, in_ny;
  int He;
  long long n_edge; // work items of the ring
  // Polls of a row copy that has not landed, after its first test, before
  // the warp gives up (flag bit 1, DVBE_ERR_TIMEOUT on the host); 0: every
  // wait gives up at once.
  unsigned long long wait_limit;

  double rho0;
  double b_phi;          // phi = delta + b (delta_eq - delta): DUGKS f_bar^+, BKG f_tilde^+,
                         // collision-free faces f^n
  double q_face;         // DUGKS face: f = f_bar + q (f_eq - f_bar)
  double dev_scale[3];   // deviation storage scale per weight class (rest, axis, diagonal)
  double fd_nux, fd_nuy; // BKG-FD: c dt / dx, c dt / dy (uniform meshes)

  // Geometry tables in compute precision (double for F64, float otherwise).
  const void *xfth, *xfs; // [nx+3]: x-face k at k+1: theta_k, h c / (xc_k - xc_{k-1})
  const void *xct, *xcu;  // [nx+2]: column i at i+1: h c / (xc_{i+1} - xc_{i-1}), dt c / dx_i
  const void *yfth, *yfs; // [ny+3]
  const void *yct, *ycu;  // [ny+2]
  double ext[4];          // ghost extrapolation factor per side (W E S N)
  const unsigned char *segid[4]; // W, E: [ny]; S, N: [nx]
  int nseg[4];
  SegParam seg[4][DVBE_MAX_SEGMENTS];

  unsigned int *flag; // bit 0: divergence seen; bit 1: a bounded wait ran out
  int walls_only;     // every non-periodic side is a bounce-back or diffuse wall
};

// Default of CaseArgs::wait_limit.
constexpr unsigned long long kDefaultWaitLimit = 1ull << 24;

// Streams of a step: the main stream, and a side stream with two events to
// run the ring kernel beside the inner kernel (fork: main -> side, join:
// side -> main).
struct StepStreams {
  cudaStream_t main, side;
  cudaEvent_t fork, join;
};

// Step launchers (one translation unit per storage mode).
cudaError_t launch_step(int store, int scheme, const CaseArgs &a, int blocks, int warps_per_block,
                        const StepStreams &ss);
cudaError_t launch_step_batch(int store, int scheme, const CaseArgs *d_cases,
                              const long long *d_prefix, int ncases, long long nitems,
                              unsigned long long *d_queue, int blocks, int warps_per_block,
                              cudaStream_t s);

// Auxiliary kernels (aux_kernels.cu).  Host-side arrays are double, unpitched.
struct FieldView {
  void *f; // storage base
  long long plane;
  int pitch, nx, ny, store;
  double rho0, scale[3], RT, tau, dt; // scale: deviation storage scale per weight class
};

// Deviation-storage scales per weight class (rest, axis, diagonal).  16-bit
// modes: the power of two nearest to dev_scale * w * rho0, so that scaling in
// and out is exact; dev_scale <= 0 selects the default (1/256 for FP16, 1 for
// BF16).  FP32 deviations are stored unscaled (a power-of-two scale changes
// no FP32 rounding) and the other modes have no scale: 1.
void deviation_scales(int precision, double dev_scale, double rho0, double out[3]);
cudaError_t aux_init_eq(const FieldView &v, const double *d_rho, const double *d_ux,
                        const double *d_uy, cudaStream_t s);
cudaError_t aux_init_ce(const FieldView &v, const double *d_rho, const double *d_ux,
                        const double *d_uy, const double *const *d_deriv, cudaStream_t s);
// f_tilde = w_alpha rho0 (fluid at rest)
cudaError_t aux_fill_rest(const FieldView &v, cudaStream_t s);
// The halo columns of every row and field (CaseArgs::hx = hx of them on each
// side; v.f addresses column 0) refreshed from the columns they copy:
// columns -hx .. -1 from nx-hx .. nx-1, columns nx .. nx+hx-1 from 0 .. hx-1.
cudaError_t aux_fill_halo(const FieldView &v, int hx, cudaStream_t s);
// one field alpha: double [ny][nx] <-> storage
cudaError_t aux_set_field(const FieldView &v, int alpha, const double *d_src, cudaStream_t s);
cudaError_t aux_get_field(const FieldView &v, int alpha, double *d_dst, cudaStream_t s);
cudaError_t aux_moments(const FieldView &v, double *d_rho, double *d_ux, double *d_uy,
                        cudaStream_t s);
// Deterministic FP64 reductions; partials must hold kReduceBlocks * 3 doubles,
// result 3 doubles.
constexpr int kReduceBlocks = 296;
// Cell volumes: d_vol_c[j * vpitch + i] when d_vol_c is not NULL (a
// quadrilateral mesh), else d_vol_x[i] * d_vol_y[j].
cudaError_t aux_conserved(const FieldView &v, const double *d_vol_x, const double *d_vol_y,
                          const double *d_vol_c, long long vpitch, double *d_partials, double *d_out,
                          cudaStream_t s);
// One line of cells (axis 0: a column over rows lo..lo+n-1, axis 1: a row
// over columns lo..lo+n-1) of all nine fields to / from a dense buffer
// [9][n] of elem-byte elements, as stored.
cudaError_t aux_copy_line(const FieldView &v, int elem, int axis, int index, int lo, int n,
                          void *buf, int to_buf, cudaStream_t s);
// sums |u - ref|^2 and |ref|^2 (mode 0: ref = given arrays, E_u); mode 1:
// residual against d_ua/d_va = previous velocity, which is then overwritten.
cudaError_t aux_velocity_error(const FieldView &v, double *d_ua, double *d_va, int mode,
                               double *d_partials, double *d_out, cudaStream_t s);

} // namespace dvbe
