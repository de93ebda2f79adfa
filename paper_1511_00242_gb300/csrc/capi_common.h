// Host-side pieces shared by the single-solver and the batched C ABI.
#pragma once

#include <string>
#include <vector>

#include "internal.h"

struct dvbe_mesh_ {
  int nx, ny;
  std::vector<double> xf, yf;   // tensor mesh: face coordinates
  bool quad = false;            // quadrilateral mesh: vertex coordinates
  std::vector<double> X, Y;     // [(ny+1)][(nx+1)]
};

namespace dvbe {

// Face tables of a quadrilateral mesh, one array of each per face (x-faces
// [ny][nx+1], y-faces [ny+1][nx]); lengths scaled by s = h c (1 for the
// central face).  L, R: the cells on either side (R on the normal's side).
enum {
  QF_TH,      // theta: the centre line crosses the face at x_L + theta d
  QF_OX,      // (x_b - x_L - theta d) / s
  QF_OY,
  QF_DX,      // d / s = (x_R - x_L) / s
  QF_DY,
  QF_TX,      // n s / (d . n): face-gradient correction direction
  QF_TY,
  QF_BX,      // (x_b - x_L) / s
  QF_BY,
  QF_NX,      // unit normal n
  QF_NY,
  QF_AX,      // n A: the flux weight of the update
  QF_AY,
  kQF
};

// Geometry of a quadrilateral mesh for the multi-pass step (quad_mesh.cu).
struct QuadHost {
  std::vector<double> jinv;     // [4][(nx+4)(ny+4)]: s J^-T of the padded cells
  std::vector<double> fx, fy;   // [kQF][faces]
  std::vector<double> vs, vol;  // [ny][nx]: dt c / |V|, |V|
  std::vector<double> ext;      // wall extrapolation: W, E [ny] each, then S, N [nx+4] each
  std::vector<unsigned char> mir; // as ext: 1 when the face normal lies along x
  std::vector<double> bn;       // outward normals (x, y): W, E [2 ny] each, then S, N [2 nx] each
  double s = 1, eshift = 1;     // length scale of the tables; 0: the central face
};

// A validated problem with its host geometry tables (double precision).
struct Problem {
  int nx = 0, ny = 0;
  std::vector<double> xf, yf;
  double RT = 0, tau = 0, dt = 0, rho0 = 1, c = 1, cfl = 0;
  double scale[3] = {1, 1, 1}; // deviation storage scale per weight class
  int user_scheme = 0, kernel = 0, store = 0;
  bool per_x = false, per_y = false;
  std::vector<dvbe_bc_segment> bc[4];
  std::vector<double> xfth, xfs, xct, xcu, yfth, yfs, yct, ycu, volx, voly;
  double ext[4] = {0, 0, 0, 0};
  std::vector<unsigned char> segid[4];
  double b_phi = 0, q_face = 0, fd_nux = 0, fd_nuy = 0; // transform coefficients (increment forms)
  double b_tp = 0;             // f_tilde^+ = f_tilde + b_tp (f_eq - f_tilde)
  int recon = 0;               // dvbe_recon
  bool multipass = false;      // multi-pass FP64 step with face arrays
  std::vector<double> xg, yg, xoff, yoff; // its gradient and foot-offset tables (MPArgs)
  bool quad = false;           // quadrilateral mesh (multi-pass step only)
  QuadHost q;
  int pitch = 0, elem = 0;
  int hx = 0;                  // halo columns of a row (CaseArgs::hx)
  long long plane = 0;
};

// Device copy of the tables (one allocation).
struct DeviceProblem {
  char *blob = nullptr;
  double *volx = nullptr, *voly = nullptr;
};

// Buffers and tables of the multi-pass step (multipass.cu), all of one
// element type: double (FP64 storage) or float (FP32 storage), elem bytes.
struct MPArgs {
  void *phi;           // [9][ny+4][nx+4]: phi with two ghost layers
  long long pplane;    // (ny+4)(nx+4)
  void *tp;            // [9][ny][nx]: f_tilde^+
  void *fx, *fy;       // [9][ny][nx+1], [9][ny+1][nx]: face distributions
  const void *xg;      // [nx+4]: cell c at c+2: h c / (x_{c+1} - x_{c-1})
  const void *yg;      // [ny+4]
  const void *xoff;    // [2(nx+1)]: face k: (x_b - x_{k-1}) / (h c), (x_b - x_k) / (h c)
  const void *yoff;    // [2(ny+1)]
  double b_tp;         // f_tilde^+ = f_tilde + b_tp (f_eq - f_tilde)
  int nx, ny, recon, scheme, elem;
  // quadrilateral mesh (QuadHost on the device); quad == 0 on tensor meshes
  int quad;
  double eshift;
  const void *jinv, *qfx, *qfy, *vs, *qext, *qbn;
  const unsigned char *qmir;
};
// Tables of a quadrilateral mesh: validates it against the boundary
// segments and fills pb.q and pb.segid.
dvbe_status quad_tables(const dvbe_mesh_ &m, Problem &pb);
double quad_min_edge(const dvbe_mesh_ &m); // shortest cell edge
cudaError_t launch_multipass(const CaseArgs &a, const MPArgs &m, cudaStream_t s);
constexpr int kMultipassKernels = 6; // launches of one multi-pass step

// Autotuner cache (tune_cache.cu): launch shapes keyed by tune_key(what),
// which appends the GPU name, SM count and library build to `what`.
struct TuneEntry {
  int strip_rows = 0, warps_per_block = 0, blocks = 0;
  double ms = 0;
};
void tune_set_path(const char *path);
std::string tune_key(const std::string &what);
bool tune_lookup(const std::string &key, TuneEntry *out);
void tune_store(const std::string &key, const TuneEntry &e);

dvbe_status fail(dvbe_status st, const std::string &msg);
dvbe_status cuda_fail(cudaError_t e, const char *what);
void *dmalloc(size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);
// halo: lay the rows out with halo columns when the mesh is periodic in x
// and the fused step runs (CaseArgs::hx).
dvbe_status build_problem(const dvbe_params *p, Problem &pb, bool halo = false);
dvbe_status upload_problem(const Problem &pb, DeviceProblem &dp, CaseArgs &a, cudaStream_t s);
void set_strips(CaseArgs &a, int H, int store);
// Kernel launches of one step (two when the inner strips run in their own kernel).
int kernels_per_step(const CaseArgs &a);
FieldView view_of(const Problem &pb, void *f);
int sm_count();
dvbe_status stage_fields(const double *const *src, int count, size_t n, cudaStream_t s,
                         double **out);
// Tensor maps of one f_tilde buffer for the step kernel's row pipeline.
dvbe_status make_tensor_maps(const Problem &pb, void *f, CUtensorMap *main_map,
                             CUtensorMap *wrap_map);

cudaError_t launch_step_f64(int scheme, const CaseArgs &a, int blocks, int wpb, const StepStreams &s);
cudaError_t launch_step_f32(int store, int scheme, const CaseArgs &a, int blocks, int wpb,
                            const StepStreams &s);
cudaError_t launch_step_f16(int store, int scheme, const CaseArgs &a, int blocks, int wpb,
                            const StepStreams &s);
int inner_blocks_per_sm_f64(int scheme, int wpb);
int inner_blocks_per_sm_f32(int store, int scheme, int wpb);
int inner_blocks_per_sm_f16(int store, int scheme, int wpb);
cudaError_t launch_batch_f64(int scheme, const CaseArgs *c, const long long *p, int n, long long ni,
                             unsigned long long *q, int blocks, int wpb, cudaStream_t s);
cudaError_t launch_batch_f32(int store, int scheme, const CaseArgs *c, const long long *p, int n,
                             long long ni, unsigned long long *q, int blocks, int wpb,
                             cudaStream_t s);
cudaError_t launch_batch_f16(int store, int scheme, const CaseArgs *c, const long long *p, int n,
                             long long ni, unsigned long long *q, int blocks, int wpb,
                             cudaStream_t s);

} // namespace dvbe
