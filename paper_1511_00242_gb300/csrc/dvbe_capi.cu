// C ABI of libdvbe (include/dvbe.h): meshes, solvers, device memory, the
// step driver with optional CUDA-graph replay, readback, reductions and the
// launch-shape autotuner.  Host code only; the kernels live in
// step_kernel.cuh (fused step) and aux_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "capi_common.h"

using namespace dvbe;

#ifndef DVBE_RING_PRIORITY
#define DVBE_RING_PRIORITY 0
#endif

// ---------------------------------------------------------------------------
// errors, allocator
// ---------------------------------------------------------------------------

namespace dvbe {

static thread_local std::string g_err;
static dvbe_alloc_fn g_alloc = nullptr;
static dvbe_free_fn g_free = nullptr;
static void *g_ctx = nullptr;

dvbe_status fail(dvbe_status st, const std::string &msg) {
  g_err = msg;
  return st;
}

dvbe_status cuda_fail(cudaError_t e, const char *what) {
  return fail(DVBE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void *dmalloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (g_alloc) return g_alloc(bytes, (void *)s, g_ctx);
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dfree(void *p, cudaStream_t s) {
  if (!p) return;
  if (g_free)
    g_free(p, (void *)s, g_ctx);
  else
    cudaFree(p);
}

cudaError_t launch_step(int store, int scheme, const CaseArgs &a, int blocks, int wpb,
                        const StepStreams &s) {
  switch (store) {
    case ST_F64:
      return launch_step_f64(scheme, a, blocks, wpb, s);
    case ST_F32:
    case ST_F32_DEV:
      return launch_step_f32(store, scheme, a, blocks, wpb, s);
    default:
      return launch_step_f16(store, scheme, a, blocks, wpb, s);
  }
}

cudaError_t launch_step_batch(int store, int scheme, const CaseArgs *c, const long long *p, int n,
                              long long ni, unsigned long long *q, int blocks, int wpb,
                              cudaStream_t s) {
  switch (store) {
    case ST_F64:
      return launch_batch_f64(scheme, c, p, n, ni, q, blocks, wpb, s);
    case ST_F32:
    case ST_F32_DEV:
      return launch_batch_f32(store, scheme, c, p, n, ni, q, blocks, wpb, s);
    default:
      return launch_batch_f16(store, scheme, c, p, n, ni, q, blocks, wpb, s);
  }
}

// ---------------------------------------------------------------------------
// problem set-up shared by the solver and the batch
// ---------------------------------------------------------------------------

void deviation_scales(int precision, double dev_scale, double rho0, double out[3]) {
  if (precision != DVBE_F16_DEV && precision != DVBE_BF16_DEV) {
    out[0] = out[1] = out[2] = 1.0;
    return;
  }
  const double sigma = dev_scale > 0 ? dev_scale : (precision == DVBE_F16_DEV ? 1.0 / 256.0 : 1.0);
  const double w[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
  for (int c = 0; c < 3; ++c) out[c] = std::exp2(std::floor(std::log2(sigma * w[c] * rho0) + 0.5));
}

static int elem_bytes(int store) {
  return store == ST_F64 ? 8 : ((store == ST_F16_DEV || store == ST_BF16_DEV) ? 2 : 4);
}

static bool uniform(const std::vector<double> &f) {
  const int n = (int)f.size() - 1;
  const double d0 = f[1] - f[0];
  for (int i = 1; i < n; ++i)
    if (std::fabs((f[i + 1] - f[i]) - d0) > 1e-12 * std::fabs(d0)) return false;
  return true;
}

static int find_seg(const std::vector<dvbe_bc_segment> &segs, double t) {
  for (size_t k = 0; k < segs.size(); ++k)
    if (t >= segs[k].s0 && t < segs[k].s1) return (int)k;
  return -1;
}

static double c_lat(const Problem &pb) { return std::sqrt(3.0 * pb.RT); }

dvbe_status build_problem(const dvbe_params *p, Problem &pb, bool halo) {
  if (!p) return fail(DVBE_ERR_INVALID_ARG, "params is NULL");
  if (!p->mesh) return fail(DVBE_ERR_INVALID_ARG, "params.mesh is NULL");
  const dvbe_mesh_ &m = *p->mesh;
  if (!(p->RT > 0) || !(p->tau > 0) || !(p->dt > 0) || !std::isfinite(p->RT) ||
      !std::isfinite(p->dt) || std::isnan(p->tau))
    return fail(DVBE_ERR_INVALID_ARG, "RT, tau and dt must be positive and finite");
  if (p->scheme < DVBE_DUGKS || p->scheme > DVBE_CFREE_CENTRAL)
    return fail(DVBE_ERR_INVALID_ARG, "unknown scheme");
  if (p->precision < DVBE_F64 || p->precision > DVBE_BF16_DEV)
    return fail(DVBE_ERR_INVALID_ARG, "unknown precision");
  pb.nx = m.nx;
  pb.ny = m.ny;
  pb.xf = m.xf;
  pb.yf = m.yf;
  pb.quad = m.quad;
  pb.RT = p->RT;
  pb.tau = p->tau;
  pb.dt = p->dt;
  pb.rho0 = p->rho0 > 0 ? p->rho0 : 1.0;
  pb.user_scheme = p->scheme;
  pb.store = p->precision;
  deviation_scales(p->precision, p->dev_scale, pb.rho0, pb.scale);
  bool per[4];
  for (int s = 0; s < 4; ++s) {
    if (p->nbc[s] < 1 || p->nbc[s] > DVBE_MAX_SEGMENTS || !p->bc[s])
      return fail(DVBE_ERR_INVALID_ARG, "each side needs 1.." + std::to_string(DVBE_MAX_SEGMENTS) +
                                            " boundary segments");
    pb.bc[s].assign(p->bc[s], p->bc[s] + p->nbc[s]);
    per[s] = false;
    for (auto &g : pb.bc[s]) {
      if (g.kind < DVBE_BC_PERIODIC || g.kind > DVBE_BC_OUTFLOW_NEQ)
        return fail(DVBE_ERR_INVALID_ARG, "unknown boundary kind");
      if (g.kind == DVBE_BC_PERIODIC) per[s] = true;
      if ((g.kind == DVBE_BC_INFLOW_EQ || g.kind == DVBE_BC_OUTFLOW_NEQ) && !(g.rho > 0))
        return fail(DVBE_ERR_INVALID_ARG, "inflow / outflow density must be positive");
    }
    if (per[s] && p->nbc[s] != 1)
      return fail(DVBE_ERR_INVALID_ARG, "a periodic side takes exactly one segment");
  }
  if (per[0] != per[1] || per[2] != per[3])
    return fail(DVBE_ERR_INVALID_ARG, "periodic must pair W with E and S with N");
  pb.per_x = per[0];
  pb.per_y = per[2];

  // Eq. eq:cfl
  double dmin = INFINITY;
  if (m.quad) {
    dmin = quad_min_edge(m);
  } else {
    for (int i = 0; i < pb.nx; ++i) dmin = std::min(dmin, pb.xf[i + 1] - pb.xf[i]);
    for (int j = 0; j < pb.ny; ++j) dmin = std::min(dmin, pb.yf[j + 1] - pb.yf[j]);
  }
  pb.cfl = pb.dt * std::sqrt(6.0 * pb.RT) / dmin;
  if (pb.cfl >= 1.0 && !p->allow_cfl_ge_1) {
    char b[160];
    snprintf(b, sizeof b, "CFL number %.6g >= 1 (dt |xi|_max / dx_min); set allow_cfl_ge_1", pb.cfl);
    return fail(DVBE_ERR_CFL, b);
  }

  pb.kernel = p->scheme == DVBE_DUGKS ? SC_DUGKS : (p->scheme == DVBE_BKG ? SC_BKG_FV : SC_CFREE);
  if (p->recon != DVBE_RECON_LINEAR && p->recon != DVBE_RECON_UPWIND_CELL)
    return fail(DVBE_ERR_INVALID_ARG, "unknown reconstruction");
  if (p->path != DVBE_PATH_FUSED && p->path != DVBE_PATH_MULTIPASS)
    return fail(DVBE_ERR_INVALID_ARG, "unknown step path");
  pb.recon = p->recon;
  pb.multipass = p->path == DVBE_PATH_MULTIPASS || p->recon == DVBE_RECON_UPWIND_CELL || m.quad;
  if (m.quad && ((p->precision != DVBE_F64 && p->precision != DVBE_F32) || p->bkg_fd))
    return fail(DVBE_ERR_UNSUPPORTED, "a quadrilateral mesh runs the multi-pass step, in FP64 or "
                                      "FP32 storage and finite-volume form only");
  if (pb.multipass && ((p->precision != DVBE_F64 && p->precision != DVBE_F32) || p->bkg_fd))
    return fail(DVBE_ERR_UNSUPPORTED, "the multi-pass step (and the upwind-cell reconstruction) runs "
                                      "in FP64 or FP32 storage and finite-volume form only");
  if (pb.recon == DVBE_RECON_UPWIND_CELL && p->scheme == DVBE_CFREE_CENTRAL)
    return fail(DVBE_ERR_UNSUPPORTED, "the central collision-free face has no upwind-cell form");
  if (p->bkg_fd) {
    if (p->scheme != DVBE_BKG || !pb.per_x || !pb.per_y || !uniform(pb.xf) || !uniform(pb.yf))
      return fail(DVBE_ERR_UNSUPPORTED,
                  "the finite-difference BKG form needs BKG on a uniform, doubly periodic mesh");
    pb.kernel = SC_BKG_FD;
  }

  // geometry (Sec 2.2 finite volumes on the tensor mesh)
  const int nx = pb.nx, ny = pb.ny;
  const double c = std::sqrt(3.0 * pb.RT), h = 0.5 * pb.dt;
  auto centres = [](const std::vector<double> &f, bool periodic, std::vector<double> &cb) {
    const int n = (int)f.size() - 1;
    cb.assign(n + 2, 0.0); // cb[i+1] = centre of cell i, i = -1..n
    for (int i = 0; i < n; ++i) cb[i + 1] = 0.5 * (f[i] + f[i + 1]);
    const double L = f[n] - f[0];
    if (periodic) {
      cb[0] = cb[n] - L;
      cb[n + 1] = cb[1] + L;
    } else {
      cb[0] = 2.0 * f[0] - cb[1];
      cb[n + 1] = 2.0 * f[n] - cb[n];
    }
  };
  std::vector<double> xcb, ycb;
  centres(pb.xf, pb.per_x, xcb);
  centres(pb.yf, pb.per_y, ycb);
  auto faces = [&](const std::vector<double> &f, const std::vector<double> &cb,
                   std::vector<double> &th, std::vector<double> &s) {
    const int n = (int)f.size() - 1;
    th.assign(n + 3, 0.5);
    s.assign(n + 3, 0.0);
    for (int k = 0; k <= n; ++k) {
      const double cl = cb[k], cr = cb[k + 1]; // centres of cells k-1, k
      th[k + 1] = (f[k] - cl) / (cr - cl);
      s[k + 1] = h * c / (cr - cl);
    }
  };
  auto cols = [&](const std::vector<double> &f, const std::vector<double> &cb,
                  std::vector<double> &t, std::vector<double> &u) {
    const int n = (int)f.size() - 1;
    t.assign(n + 2, 0.0);
    u.assign(n + 2, 0.0);
    for (int i = 0; i < n; ++i) {
      t[i + 1] = h * c / (cb[i + 2] - cb[i]);
      u[i + 1] = pb.dt * c / (f[i + 1] - f[i]);
    }
  };
  faces(pb.xf, xcb, pb.xfth, pb.xfs);
  faces(pb.yf, ycb, pb.yfth, pb.yfs);
  cols(pb.xf, xcb, pb.xct, pb.xcu);
  cols(pb.yf, ycb, pb.yct, pb.ycu);
  if (p->scheme == DVBE_CFREE_CENTRAL) {
    // Eq. cfd1: the face value at x_b itself, no shift along the
    // characteristic: normal and tangential slope factors vanish
    std::fill(pb.xfs.begin(), pb.xfs.end(), 0.0);
    std::fill(pb.yfs.begin(), pb.yfs.end(), 0.0);
    std::fill(pb.xct.begin(), pb.xct.end(), 0.0);
    std::fill(pb.yct.begin(), pb.yct.end(), 0.0);
  }
  pb.ext[0] = (xcb[0] - xcb[1]) / (xcb[1] - xcb[2]);
  pb.ext[1] = (xcb[nx + 1] - xcb[nx]) / (xcb[nx] - xcb[nx - 1]);
  pb.ext[2] = (ycb[0] - ycb[1]) / (ycb[1] - ycb[2]);
  pb.ext[3] = (ycb[ny + 1] - ycb[ny]) / (ycb[ny] - ycb[ny - 1]);
  pb.volx.resize(nx);
  pb.voly.resize(ny);
  for (int i = 0; i < nx; ++i) pb.volx[i] = pb.xf[i + 1] - pb.xf[i];
  for (int j = 0; j < ny; ++j) pb.voly[j] = pb.yf[j + 1] - pb.yf[j];
  // segment of each boundary face by its centre coordinate
  for (int s = 0; s < 4; ++s) {
    const bool xs = s < 2;
    const int n = xs ? ny : nx;
    pb.segid[s].assign(n, 0);
    if (per[s] || m.quad) continue; // quadrilateral meshes: by face midpoint (quad_tables)
    for (int k = 0; k < n; ++k) {
      const double t = xs ? ycb[k + 1] : xcb[k + 1];
      int g = find_seg(pb.bc[s], t);
      if (g < 0) return fail(DVBE_ERR_INVALID_ARG, "a boundary face is not covered by any segment");
      if (pb.bc[s][g].kind == DVBE_BC_PERIODIC)
        return fail(DVBE_ERR_INVALID_ARG, "periodic segment on a non-periodic side");
      pb.segid[s][k] = (unsigned char)g;
    }
    if ((pb.bc[s][0].kind == DVBE_BC_WALL_BOUNCEBACK || pb.bc[s][0].kind == DVBE_BC_WALL_DIFFUSE) &&
        (xs ? nx : ny) < 2)
      return fail(DVBE_ERR_INVALID_ARG, "walls need two cells normal to the side");
  }
  // transform coefficients (closed forms of Eqs. eq_trans_2 and the
  // f_tilde / f_tilde^+ transforms of Sec 2.2)
  const double tau = pb.tau, dt = pb.dt;
  pb.c = c;
  // increment forms phi = f_tilde + b (f_eq - f_tilde), f = f_bar + q (f_eq - f_bar)
  if (pb.user_scheme == DVBE_DUGKS)
    pb.b_phi = 3 * h / (2 * tau + dt); // f_bar^+ = ((2 tau - h) f_tilde + 3 h f_eq) / (2 tau + dt)
  else if (pb.kernel == SC_CFREE)
    pb.b_phi = dt / (2 * tau + dt); // the cell f^n = (2 tau f_tilde + dt f_eq) / (2 tau + dt)
  else
    pb.b_phi = 2 * dt / (2 * tau + dt); // f_tilde^+ = ((2 tau - dt) f_tilde + 2 dt f_eq) / (2 tau + dt)
  pb.q_face = h / (2 * tau + h);        // f = (2 tau f_bar + h f_eq) / (2 tau + h)
  pb.b_tp = 2 * dt / (2 * tau + dt);    // f_tilde^+ of every scheme
  if (m.quad) {
    dvbe_status st = quad_tables(m, pb);
    if (st != DVBE_OK) return st;
  }
  if (pb.multipass) {
    // cell centres c = -2 .. n+1 (periodic: shifted images; otherwise the
    // mirror ghost at -1 and n, unused beyond), the central-difference factor
    // h c / (x_{c+1} - x_{c-1}) of cells -1 .. n, and the offsets of each
    // face from its two cells' centres, over h c
    auto tables = [&](const std::vector<double> &f, const std::vector<double> &cb, bool periodic,
                      std::vector<double> &g, std::vector<double> &off) {
      const int n = (int)f.size() - 1;
      const double L = f[n] - f[0];
      std::vector<double> x(n + 4, 0.0); // x[c+2]
      for (int c = -1; c <= n; ++c) x[c + 2] = cb[c + 1];
      x[0] = periodic ? cb[n - 1] - L : 2 * x[1] - x[2];
      x[n + 3] = periodic ? cb[2] + L : 2 * x[n + 2] - x[n + 1];
      g.assign(n + 4, 0.0);
      if (p->scheme != DVBE_CFREE_CENTRAL)
        for (int c = -1; c <= n; ++c) g[c + 2] = h * c_lat(pb) / (x[c + 3] - x[c + 1]);
      off.assign(2 * (n + 1), 0.0);
      for (int k = 0; k <= n; ++k) {
        off[2 * k] = (f[k] - x[k + 1]) / (h * c_lat(pb));
        off[2 * k + 1] = (f[k] - x[k + 2]) / (h * c_lat(pb));
      }
    };
    tables(pb.xf, xcb, pb.per_x, pb.xg, pb.xoff);
    tables(pb.yf, ycb, pb.per_y, pb.yg, pb.yoff);
  }
  pb.fd_nux = c * dt / (pb.xf[1] - pb.xf[0]);
  pb.fd_nuy = c * dt / (pb.yf[1] - pb.yf[0]);
  // storage layout: rows padded to 128 bytes and at least 64 elements, so a
  // staged row box (at most 40 elements) always fits inside a row
  const int eb = elem_bytes(pb.store);
  const int align = 128 / eb;
  // halo columns (CaseArgs::hx): one 16-byte group on each side, so that the
  // row copies stay aligned; a lane's columns must not straddle the end of
  // the row, and the two copies must not overlap
  pb.hx = 0;
  if (halo && DVBE_HALO && pb.per_x && !pb.multipass && nx % lane_cols(pb.store) == 0 && nx >= 2 * (16 / eb))
    pb.hx = 16 / eb;
  pb.pitch = std::max(((nx + 2 * pb.hx + align - 1) / align) * align, 64);
  pb.plane = (long long)pb.pitch * ny;
  pb.elem = eb;
  // the step kernel addresses f_tilde with 32-bit element offsets
  if (9 * pb.plane >= (1LL << 32))
    return fail(DVBE_ERR_UNSUPPORTED, "mesh too large for one solver (9 x cells must stay below 2^32)");
  return DVBE_OK;
}

// Device copy of the geometry tables in compute precision.
template <typename Real>
static void pack_tables(const Problem &pb, std::vector<char> &blob, size_t off[8]) {
  const std::vector<double> *src[8] = {&pb.xfth, &pb.xfs, &pb.xct, &pb.xcu,
                                       &pb.yfth, &pb.yfs, &pb.yct, &pb.ycu};
  size_t pos = 0;
  for (int q = 0; q < 8; ++q) {
    off[q] = pos;
    pos += ((src[q]->size() * sizeof(Real) + 255) / 256) * 256;
  }
  blob.assign(pos, 0);
  for (int q = 0; q < 8; ++q) {
    Real *d = (Real *)(blob.data() + off[q]);
    for (size_t k = 0; k < src[q]->size(); ++k) d[k] = (Real)(*src[q])[k];
  }
}

dvbe_status upload_problem(const Problem &pb, DeviceProblem &dp, CaseArgs &a, cudaStream_t s) {
  std::vector<char> blob;
  size_t off[8];
  if (pb.store == ST_F64)
    pack_tables<double>(pb, blob, off);
  else
    pack_tables<float>(pb, blob, off);
  const size_t segbytes = 2 * (size_t)pb.ny + 2 * (size_t)pb.nx;
  const size_t volbytes = sizeof(double) * (size_t)(pb.nx + pb.ny);
  const size_t total = blob.size() + segbytes + volbytes + 256;
  dp.blob = (char *)dmalloc(total, s);
  if (!dp.blob) return fail(DVBE_ERR_OOM, "device allocation of geometry tables failed");
  std::vector<char> host(total, 0);
  memcpy(host.data(), blob.data(), blob.size());
  size_t pos = blob.size();
  size_t segoff[4];
  for (int q = 0; q < 4; ++q) {
    segoff[q] = pos;
    memcpy(host.data() + pos, pb.segid[q].data(), pb.segid[q].size());
    pos += pb.segid[q].size();
  }
  pos = ((pos + 7) / 8) * 8;
  size_t voloff = pos;
  memcpy(host.data() + pos, pb.volx.data(), sizeof(double) * pb.nx);
  memcpy(host.data() + pos + sizeof(double) * pb.nx, pb.voly.data(), sizeof(double) * pb.ny);
  cudaError_t e = cudaMemcpyAsync(dp.blob, host.data(), total, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "upload of geometry tables");
  dp.volx = (double *)(dp.blob + voloff);
  dp.voly = dp.volx + pb.nx;

  memset(&a, 0, sizeof(a));
  a.wait_limit = kDefaultWaitLimit;
  a.plane = pb.plane;
  a.pitch = pb.pitch;
  a.hx = pb.hx;
  a.walls_only = DVBE_WALLS_PATH;
  for (int q = 0; q < 4; ++q)
    for (const dvbe_bc_segment &g : pb.bc[q])
      if (g.kind != DVBE_BC_PERIODIC && g.kind != DVBE_BC_WALL_BOUNCEBACK && g.kind != DVBE_BC_WALL_DIFFUSE)
        a.walls_only = 0;
  a.nx = pb.nx;
  a.ny = pb.ny;
  a.per_x = pb.per_x;
  a.per_y = pb.per_y;
  a.rho0 = pb.rho0;
  a.b_phi = pb.b_phi;
  a.q_face = pb.q_face;
  for (int c = 0; c < 3; ++c) a.dev_scale[c] = pb.scale[c];
  a.fd_nux = pb.fd_nux;
  a.fd_nuy = pb.fd_nuy;
  a.xfth = dp.blob + off[0];
  a.xfs = dp.blob + off[1];
  a.xct = dp.blob + off[2];
  a.xcu = dp.blob + off[3];
  a.yfth = dp.blob + off[4];
  a.yfs = dp.blob + off[5];
  a.yct = dp.blob + off[6];
  a.ycu = dp.blob + off[7];
  for (int q = 0; q < 4; ++q) {
    a.ext[q] = pb.ext[q];
    a.segid[q] = (const unsigned char *)(dp.blob + segoff[q]);
    a.nseg[q] = (int)pb.bc[q].size();
    for (size_t g = 0; g < pb.bc[q].size(); ++g) {
      a.seg[q][g].kind = pb.bc[q][g].kind;
      a.seg[q][g].rho = pb.bc[q][g].rho;
      a.seg[q][g].ux = pb.bc[q][g].ux / pb.c;
      a.seg[q][g].uy = pb.bc[q][g].uy / pb.c;
    }
  }
  return DVBE_OK;
}

void set_strips(CaseArgs &a, int H, int store) {
  const int cols = strip_cols(store);
  a.H = H;
  a.strips_x = (a.nx + cols - 1) / cols;
  a.strips_y = (a.ny + H - 1) / H;
  // Inner strips: sx >= 1 with (sx + 1) cols <= nx - 1 and sy >= 1 with
  // (sy + 1) H <= ny - 1, so that the strip's columns i0 - 1 .. i0 + cols
  // and rows j0 - 1 .. j0 + H are all cells of the mesh.
  // On a mesh periodic in y every strip row qualifies (rows wrap).
  const int sxmax = a.nx - 1 - cols >= 0 ? (a.nx - 1 - cols) / cols : 0;
  const int symax = (a.ny - 1) / H - 1;
  a.in_x0 = 1;
  a.in_nx = std::max(0, sxmax);
  if (a.hx > 0) { // halo columns: every column strip reads its wrap neighbours as cells
    a.in_x0 = 0;
    a.in_nx = a.strips_x;
  }
  a.in_y0 = a.per_y ? 0 : 1;
  a.in_ny = a.per_y ? a.strips_y : std::max(0, symax);
  a.He = H;
  a.n_edge = 0;
  if (a.in_nx == 0 || a.in_ny == 0) {
    a.in_nx = a.in_ny = 0; // one kernel over every strip
    return;
  }
  // the ring in pieces of He rows: the largest divisor of H in 4..8 below H
  for (int d = 8; d >= 4; --d)
    if (d < H && H % d == 0) {
      a.He = d;
      break;
    }
  const long long pieces_y = (a.ny + a.He - 1) / a.He;
  const long long r0 = (long long)a.in_y0 * (H / a.He);
  const long long r1 = std::min((long long)(a.in_y0 + a.in_ny) * (H / a.He), pieces_y);
  a.n_edge = (long long)a.strips_x * pieces_y - (long long)a.in_nx * (r1 - r0);
}

int kernels_per_step(const CaseArgs &a) {
  return (long long)a.in_nx * a.in_ny == 0 ? 1 : (a.n_edge > 0 ? 2 : 1);
}

FieldView view_of(const Problem &pb, void *f) {
  FieldView v;
  v.f = (char *)f + (size_t)pb.hx * pb.elem; // column 0 of row 0 of field 0
  v.plane = pb.plane;
  v.pitch = pb.pitch;
  v.nx = pb.nx;
  v.ny = pb.ny;
  v.store = pb.store;
  v.rho0 = pb.rho0;
  for (int c = 0; c < 3; ++c) v.scale[c] = pb.scale[c];
  v.RT = pb.RT;
  v.tau = pb.tau;
  v.dt = pb.dt;
  return v;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

dvbe_status make_tensor_maps(const Problem &pb, void *f, CUtensorMap *main_map,
                             CUtensorMap *wrap_map) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return fail(DVBE_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  CUtensorMapDataType dt;
  switch (pb.store) {
    case ST_F64:
      dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
      break;
    case ST_F16_DEV:
      dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
      break;
    case ST_BF16_DEV:
      dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
      break;
    default:
      dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  }
  const int es = pb.elem;
  // columns per staged row of the step kernel
  const cuuint32_t W = (cuuint32_t)stage_cols(es, lane_cols(pb.store));
  const cuuint64_t dims[3] = {(cuuint64_t)pb.pitch, (cuuint64_t)pb.ny, 9};
  const cuuint64_t strides[2] = {(cuuint64_t)pb.pitch * es, (cuuint64_t)pb.plane * es};
  const cuuint32_t box_main[3] = {W, 1, 9};
  const cuuint32_t box_wrap[3] = {(cuuint32_t)(16 / es), 1, 9};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(main_map, dt, 3, f, dims, strides, box_main, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r == CUDA_SUCCESS)
    r = enc(wrap_map, dt, 3, f, dims, strides, box_wrap, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(DVBE_ERR_CUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return DVBE_OK;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 1;
    }
  }
  return n;
}

// Upload host float64 fields (each n doubles) into one staging allocation.
dvbe_status stage_fields(const double *const *src, int count, size_t n, cudaStream_t s,
                         double **out) {
  double *d = (double *)dmalloc(sizeof(double) * n * count, s);
  if (!d) return fail(DVBE_ERR_OOM, "device staging allocation failed");
  for (int q = 0; q < count; ++q) {
    cudaError_t e = cudaMemcpyAsync(d + q * n, src[q], sizeof(double) * n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      dfree(d, s);
      return cuda_fail(e, "host to device copy");
    }
  }
  *out = d;
  return DVBE_OK;
}

} // namespace dvbe

// ---------------------------------------------------------------------------
// solver
// ---------------------------------------------------------------------------

struct dvbe_solver_ {
  Problem pb;
  DeviceProblem dp;
  CaseArgs args;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  StepStreams ss{}; // main = stream; side stream and fork / join events of the two-kernel step
  MPArgs mp{};      // multi-pass step: buffers and tables (one allocation), when used
  char *mpblob = nullptr;
  const double *qvol = nullptr; // cell volumes of a quadrilateral mesh (in mpblob)
  void *f[2] = {nullptr, nullptr};
  int cur = 0;
  unsigned *flag = nullptr;
  double *red = nullptr;  // reduction partials + 3 results
  double *uprev = nullptr; // 2 * nx * ny (residual)
  bool have_prev = false;
  dvbe_launch launch{64, 4, 0, 0};
  long long steps = 0, launches = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_len = 0;
  CUtensorMap tm[2][2]; // [buffer][main, wrap]
};

// Buffers and tables of the multi-pass step in one device allocation, in
// the storage's element type (the cell volumes of a quadrilateral mesh stay
// FP64, for the conserved sums).
static dvbe_status alloc_multipass(dvbe_solver s) {
  const Problem &pb = s->pb;
  const long long nx = pb.nx, ny = pb.ny;
  const long long pplane = (nx + 4) * (ny + 4);
  const size_t es = (size_t)pb.elem;
  // buffers, the tensor tables, then the quadrilateral-mesh tables (empty
  // on tensor meshes); the FP64 volumes and the mirror flags (bytes) last
  const QuadHost &qh = pb.q;
  const std::vector<double> *tab[10] = {&pb.xg, &pb.yg, &pb.xoff, &pb.yoff, &qh.jinv,
                                        &qh.fx, &qh.fy, &qh.vs, &qh.ext, &qh.bn};
  size_t bytes[16] = {es * 9 * pplane, es * 9 * nx * ny, es * 9 * (nx + 1) * ny, es * 9 * nx * (ny + 1)};
  for (int q = 0; q < 10; ++q) bytes[4 + q] = es * tab[q]->size();
  bytes[14] = sizeof(double) * qh.vol.size();
  bytes[15] = qh.mir.size();
  size_t off[16], total = 0;
  for (int q = 0; q < 16; ++q) {
    off[q] = total;
    total += (bytes[q] + 255) / 256 * 256;
  }
  s->mpblob = (char *)dmalloc(total, s->stream);
  if (!s->mpblob) return fail(DVBE_ERR_OOM, "device allocation of the multi-pass buffers failed");
  std::vector<char> host(total - off[4], 0);
  for (int q = 0; q < 10; ++q) {
    char *dst = host.data() + (off[4 + q] - off[4]);
    const std::vector<double> &v = *tab[q];
    if (es == 8)
      memcpy(dst, v.data(), sizeof(double) * v.size());
    else
      for (size_t k = 0; k < v.size(); ++k) ((float *)dst)[k] = (float)v[k];
  }
  if (!qh.vol.empty()) memcpy(host.data() + (off[14] - off[4]), qh.vol.data(), bytes[14]);
  if (!qh.mir.empty()) memcpy(host.data() + (off[15] - off[4]), qh.mir.data(), bytes[15]);
  cudaError_t e = cudaMemsetAsync(s->mpblob, 0, off[4], s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->mpblob + off[4], host.data(), host.size(), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "multi-pass set-up");
  MPArgs &m = s->mp;
  m.phi = s->mpblob + off[0];
  m.pplane = pplane;
  m.tp = s->mpblob + off[1];
  m.fx = s->mpblob + off[2];
  m.fy = s->mpblob + off[3];
  m.xg = s->mpblob + off[4];
  m.yg = s->mpblob + off[5];
  m.xoff = s->mpblob + off[6];
  m.yoff = s->mpblob + off[7];
  m.b_tp = pb.b_tp;
  m.nx = pb.nx;
  m.ny = pb.ny;
  m.recon = pb.recon;
  m.scheme = pb.kernel;
  m.elem = pb.elem;
  m.quad = pb.quad ? 1 : 0;
  m.eshift = qh.eshift;
  m.jinv = s->mpblob + off[8];
  m.qfx = s->mpblob + off[9];
  m.qfy = s->mpblob + off[10];
  m.vs = s->mpblob + off[11];
  m.qext = s->mpblob + off[12];
  m.qbn = s->mpblob + off[13];
  s->qvol = (const double *)(s->mpblob + off[14]);
  m.qmir = (const unsigned char *)(s->mpblob + off[15]);
  return DVBE_OK;
}

static void drop_graphs(dvbe_solver s) {
  for (int p = 0; p < 2; ++p)
    if (s->graph[p]) {
      cudaGraphExecDestroy(s->graph[p]);
      s->graph[p] = nullptr;
    }
  s->graph_len = 0;
}

static FieldView cur_view(dvbe_solver s) { return view_of(s->pb, s->f[s->cur]); }

extern "C" {

const char *dvbe_last_error(void) { return g_err.c_str(); }

const char *dvbe_version(void) { return "libdvbe 0.1 sm_103a"; }

dvbe_status dvbe_set_allocator(dvbe_alloc_fn alloc, dvbe_free_fn free_, void *ctx) {
  if ((alloc == nullptr) != (free_ == nullptr))
    return fail(DVBE_ERR_INVALID_ARG, "allocator and free must both be set or both be NULL");
  g_alloc = alloc;
  g_free = free_;
  g_ctx = ctx;
  return DVBE_OK;
}

dvbe_status dvbe_d2q9(double RT, double *xi, double *w, int *opp) {
  if (!(RT > 0) || !xi || !w || !opp) return fail(DVBE_ERR_INVALID_ARG, "bad argument");
  const double c = std::sqrt(3.0 * RT);
  static const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  static const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  static const int op[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
  for (int a = 0; a < 9; ++a) {
    xi[2 * a] = c * ex[a];
    xi[2 * a + 1] = c * ey[a];
    w[a] = a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    opp[a] = op[a];
  }
  return DVBE_OK;
}

dvbe_status dvbe_mesh_create(int nx, int ny, const double *xf, const double *yf, dvbe_mesh *out) {
  if (!out || !xf || !yf) return fail(DVBE_ERR_INVALID_ARG, "NULL pointer");
  *out = nullptr;
  if (nx < 2 || ny < 2) return fail(DVBE_ERR_INVALID_ARG, "nx and ny must be >= 2");
  if ((long long)nx * ny > (1LL << 31)) return fail(DVBE_ERR_INVALID_ARG, "mesh too large");
  for (int i = 0; i < nx; ++i)
    if (!(xf[i + 1] > xf[i]) || !std::isfinite(xf[i + 1]))
      return fail(DVBE_ERR_INVALID_ARG, "x faces must be finite and strictly increasing");
  for (int j = 0; j < ny; ++j)
    if (!(yf[j + 1] > yf[j]) || !std::isfinite(yf[j + 1]))
      return fail(DVBE_ERR_INVALID_ARG, "y faces must be finite and strictly increasing");
  dvbe_mesh m = new (std::nothrow) dvbe_mesh_;
  if (!m) return fail(DVBE_ERR_OOM, "host allocation failed");
  m->nx = nx;
  m->ny = ny;
  m->xf.assign(xf, xf + nx + 1);
  m->yf.assign(yf, yf + ny + 1);
  *out = m;
  return DVBE_OK;
}

void dvbe_mesh_destroy(dvbe_mesh mesh) { delete mesh; }

dvbe_status dvbe_mesh_geometry(dvbe_mesh m, double *xc, double *yc, double *vol) {
  if (!m) return fail(DVBE_ERR_INVALID_ARG, "NULL mesh");
  if (m->quad)
    return fail(DVBE_ERR_UNSUPPORTED, "a quadrilateral mesh has no face coordinates: use dvbe_mesh_cells");
  for (int i = 0; i < m->nx && xc; ++i) xc[i] = 0.5 * (m->xf[i] + m->xf[i + 1]);
  for (int j = 0; j < m->ny && yc; ++j) yc[j] = 0.5 * (m->yf[j] + m->yf[j + 1]);
  if (vol)
    for (int j = 0; j < m->ny; ++j)
      for (int i = 0; i < m->nx; ++i)
        vol[(size_t)j * m->nx + i] = (m->xf[i + 1] - m->xf[i]) * (m->yf[j + 1] - m->yf[j]);
  return DVBE_OK;
}

dvbe_status dvbe_faces_uniform(int n, double a, double b, double *out) {
  if (n < 1 || !(b > a) || !out) return fail(DVBE_ERR_INVALID_ARG, "bad argument");
  for (int i = 0; i <= n; ++i) out[i] = a + (b - a) * (double)i / (double)n;
  return DVBE_OK;
}

dvbe_status dvbe_faces_tanh(int n, double a, double b, double beta, double *out) {
  if (n < 1 || !(b > a) || !(beta > 0) || !out) return fail(DVBE_ERR_INVALID_ARG, "bad argument");
  const double tb = std::tanh(beta);
  for (int i = 0; i <= n; ++i) {
    const double s = (double)i / (double)n;
    out[i] = a + (b - a) * 0.5 * (1.0 + std::tanh(beta * (2.0 * s - 1.0)) / tb);
  }
  return DVBE_OK;
}

dvbe_status dvbe_faces_geometric(int n, double a, double d0, double ratio, double *out) {
  if (n < 1 || !(d0 > 0) || !(ratio > 0) || !out) return fail(DVBE_ERR_INVALID_ARG, "bad argument");
  for (int i = 0; i <= n; ++i)
    out[i] = ratio == 1.0 ? a + d0 * i : a + d0 * (std::pow(ratio, (double)i) - 1.0) / (ratio - 1.0);
  return DVBE_OK;
}

dvbe_status dvbe_dt_from_cfl(dvbe_mesh m, double RT, double cfl, double *dt) {
  if (!m || !(RT > 0) || !(cfl > 0) || !dt) return fail(DVBE_ERR_INVALID_ARG, "bad argument");
  double dmin = INFINITY;
  if (m->quad) {
    dmin = quad_min_edge(*m);
  } else {
    for (int i = 0; i < m->nx; ++i) dmin = std::min(dmin, m->xf[i + 1] - m->xf[i]);
    for (int j = 0; j < m->ny; ++j) dmin = std::min(dmin, m->yf[j + 1] - m->yf[j]);
  }
  *dt = cfl * dmin / (std::sqrt(6.0) * std::sqrt(RT));
  return DVBE_OK;
}

void dvbe_solver_destroy(dvbe_solver s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  drop_graphs(s);
  dfree(s->f[0], s->stream);
  dfree(s->f[1], s->stream);
  dfree(s->flag, s->stream);
  dfree(s->red, s->stream);
  dfree(s->uprev, s->stream);
  dfree(s->dp.blob, s->stream);
  dfree(s->mpblob, s->stream);
  if (s->ss.side) cudaStreamDestroy(s->ss.side);
  if (s->ss.fork) cudaEventDestroy(s->ss.fork);
  if (s->ss.join) cudaEventDestroy(s->ss.join);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
}

dvbe_status dvbe_solver_create(const dvbe_params *p, dvbe_solver *out) {
  if (!out) return fail(DVBE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  dvbe_solver s = new (std::nothrow) dvbe_solver_;
  if (!s) return fail(DVBE_ERR_OOM, "host allocation failed");
  dvbe_status st = build_problem(p, s->pb, true);
  if (st != DVBE_OK) {
    delete s;
    return st;
  }
  if (p->cuda_stream) {
    s->stream = (cudaStream_t)p->cuda_stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete s;
      return cuda_fail(e, "cudaStreamCreate");
    }
    s->own_stream = true;
  }
  s->ss.main = s->stream;
  {
    // DVBE_RING_PRIORITY 1: the ring kernel's stream at the highest priority
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess)
      e = cudaStreamCreateWithPriority(&s->ss.side, cudaStreamNonBlocking,
                                       DVBE_RING_PRIORITY ? greatest : least);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ss.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ss.join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      dvbe_solver_destroy(s);
      return cuda_fail(e, "side stream of the step");
    }
  }
  st = upload_problem(s->pb, s->dp, s->args, s->stream);
  const size_t fbytes = (size_t)s->pb.plane * 9 * s->pb.elem;
  if (st == DVBE_OK) {
    s->f[0] = dmalloc(fbytes, s->stream);
    s->f[1] = dmalloc(fbytes, s->stream);
    s->flag = (unsigned *)dmalloc(sizeof(unsigned), s->stream);
    s->red = (double *)dmalloc(sizeof(double) * (kReduceBlocks * 3 + 3), s->stream);
    if (!s->f[0] || !s->f[1] || !s->flag || !s->red) st = fail(DVBE_ERR_OOM, "device allocation of f_tilde failed");
  }
  for (int p = 0; p < 2 && st == DVBE_OK; ++p)
    st = make_tensor_maps(s->pb, s->f[p], &s->tm[p][0], &s->tm[p][1]);
  if (st == DVBE_OK && s->pb.multipass) st = alloc_multipass(s);
  if (st == DVBE_OK) {
    cudaError_t e = cudaMemsetAsync(s->f[0], 0, fbytes, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->f[1], 0, fbytes, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->flag, 0, sizeof(unsigned), s->stream);
    if (e == cudaSuccess) e = aux_fill_rest(cur_view(s), s->stream);
    s->launches += 1;
    if (e == cudaSuccess && s->pb.hx > 0) {
      e = aux_fill_halo(cur_view(s), s->pb.hx, s->stream);
      s->launches += 1;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "solver initialisation");
  }
  if (st != DVBE_OK) {
    dvbe_solver_destroy(s);
    return st;
  }
  s->args.flag = s->flag;
  set_strips(s->args, s->launch.strip_rows, s->pb.store);
  *out = s;
  return DVBE_OK;
}

static dvbe_status after_init(dvbe_solver s, cudaError_t e, const char *what) {
  if (e == cudaSuccess && s->pb.hx > 0) { // the halo copies of the new state
    e = aux_fill_halo(cur_view(s), s->pb.hx, s->stream);
    s->launches += 1;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, what);
  s->steps = 0;
  s->have_prev = false;
  unsigned z = 0;
  e = cudaMemcpy(s->flag, &z, sizeof z, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, what);
  return DVBE_OK;
}

dvbe_status dvbe_init_equilibrium(dvbe_solver s, const double *rho, const double *ux,
                                  const double *uy) {
  if (!s || !rho || !ux || !uy) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  const size_t n = (size_t)s->pb.nx * s->pb.ny;
  const double *src[3] = {rho, ux, uy};
  double *d = nullptr;
  dvbe_status st = stage_fields(src, 3, n, s->stream, &d);
  if (st != DVBE_OK) return st;
  cudaError_t e = aux_init_eq(cur_view(s), d, d + n, d + 2 * n, s->stream);
  s->launches += 1;
  st = after_init(s, e, "init_equilibrium");
  dfree(d, s->stream);
  return st;
}

dvbe_status dvbe_init_chapman_enskog(dvbe_solver s, const double *rho, const double *ux,
                                     const double *uy, const double *const *dd) {
  if (!s || !rho || !ux || !uy || !dd) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  for (int q = 0; q < 9; ++q)
    if (!dd[q]) return fail(DVBE_ERR_INVALID_ARG, "NULL derivative array");
  const size_t n = (size_t)s->pb.nx * s->pb.ny;
  const double *src[12] = {rho, ux, uy, dd[0], dd[1], dd[2], dd[3], dd[4], dd[5], dd[6], dd[7], dd[8]};
  double *d = nullptr;
  dvbe_status st = stage_fields(src, 12, n, s->stream, &d);
  if (st != DVBE_OK) return st;
  const double *dp[9];
  for (int q = 0; q < 9; ++q) dp[q] = d + (3 + q) * n;
  cudaError_t e = aux_init_ce(cur_view(s), d, d + n, d + 2 * n, dp, s->stream);
  s->launches += 1;
  st = after_init(s, e, "init_chapman_enskog");
  dfree(d, s->stream);
  return st;
}

dvbe_status dvbe_init_f(dvbe_solver s, const double *ft) {
  if (!s || !ft) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  const size_t n = (size_t)s->pb.nx * s->pb.ny;
  double *d = (double *)dmalloc(sizeof(double) * n, s->stream);
  if (!d) return fail(DVBE_ERR_OOM, "device staging allocation failed");
  cudaError_t e = cudaSuccess;
  for (int a = 0; a < 9 && e == cudaSuccess; ++a) {
    e = cudaMemcpyAsync(d, ft + a * n, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = aux_set_field(cur_view(s), a, d, s->stream);
    s->launches += 1;
  }
  dvbe_status st = after_init(s, e, "init_f");
  dfree(d, s->stream);
  return st;
}

dvbe_status dvbe_get_f(dvbe_solver s, double *ft) {
  if (!s || !ft) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  const size_t n = (size_t)s->pb.nx * s->pb.ny;
  double *d = (double *)dmalloc(sizeof(double) * n, s->stream);
  if (!d) return fail(DVBE_ERR_OOM, "device staging allocation failed");
  cudaError_t e = cudaSuccess;
  for (int a = 0; a < 9 && e == cudaSuccess; ++a) {
    e = aux_get_field(cur_view(s), a, d, s->stream);
    s->launches += 1;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ft + a * n, d, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  dfree(d, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "get_f");
  return DVBE_OK;
}

// Kernel launches of one step of this solver.
static int step_launches(dvbe_solver s) {
  return s->pb.multipass ? kMultipassKernels : kernels_per_step(s->args);
}

static cudaError_t launch_one(dvbe_solver s) {
  s->args.tm_main = s->tm[s->cur][0];
  s->args.tm_wrap = s->tm[s->cur][1];
  s->args.fin = s->f[s->cur];
  s->args.fout = s->f[1 - s->cur];
  cudaError_t e = s->pb.multipass ? launch_multipass(s->args, s->mp, s->stream)
                                  : launch_step(s->pb.store, s->pb.kernel, s->args, s->launch.blocks,
                                                s->launch.warps_per_block, s->ss);
  s->cur ^= 1;
  s->steps += 1;
  s->launches += step_launches(s);
  return e;
}

static cudaError_t capture(dvbe_solver s, int parity, int len) {
  cudaGraph_t g = nullptr;
  const int saved_cur = s->cur;
  const long long saved_steps = s->steps, saved_l = s->launches;
  s->cur = parity;
  cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < len; ++k) {
    cudaError_t x = launch_one(s);
    if (x != cudaSuccess && le == cudaSuccess) le = x;
  }
  e = cudaStreamEndCapture(s->stream, &g);
  s->cur = saved_cur;
  s->steps = saved_steps;
  s->launches = saved_l;
  if (le != cudaSuccess) e = le;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&s->graph[parity], g, 0);
  if (g) cudaGraphDestroy(g);
  return e;
}

dvbe_status dvbe_step_async(dvbe_solver s, long long nsteps) {
  if (!s || nsteps < 0) return fail(DVBE_ERR_INVALID_ARG, "bad argument");
  cudaError_t e = cudaSuccess;
  int chunk = s->launch.graph_chunk;
  if (chunk > 0) chunk += chunk & 1; // even, so a replay keeps the buffer parity
  if (chunk > 0 && nsteps >= chunk) {
    if (s->graph_len != chunk) {
      drop_graphs(s);
      for (int p = 0; p < 2 && e == cudaSuccess; ++p) e = capture(s, p, chunk);
      if (e != cudaSuccess) {
        drop_graphs(s);
        return cuda_fail(e, "graph capture");
      }
      s->graph_len = chunk;
    }
    while (nsteps >= chunk && e == cudaSuccess) {
      e = cudaGraphLaunch(s->graph[s->cur], s->stream);
      s->steps += chunk;
      s->launches += (long long)chunk * step_launches(s);
      nsteps -= chunk;
    }
  }
  for (long long k = 0; k < nsteps && e == cudaSuccess; ++k) e = launch_one(s);
  if (e != cudaSuccess) return cuda_fail(e, "step launch");
  return DVBE_OK;
}

dvbe_status dvbe_sync(dvbe_solver s) {
  if (!s) return fail(DVBE_ERR_INVALID_ARG, "NULL solver");
  unsigned flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, s->flag, sizeof flag, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "synchronise");
  if (flag & 2u) return fail(DVBE_ERR_TIMEOUT, "a bounded wait in the step kernel ran out");
  if (flag & 1u) return fail(DVBE_ERR_DIVERGED, "non-finite or non-positive density met");
  return DVBE_OK;
}

dvbe_status dvbe_step(dvbe_solver s, long long nsteps) {
  dvbe_status st = dvbe_step_async(s, nsteps);
  if (st != DVBE_OK) return st;
  return dvbe_sync(s);
}

dvbe_status dvbe_step_count(dvbe_solver s, long long *n) {
  if (!s || !n) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  *n = s->steps;
  return DVBE_OK;
}

dvbe_status dvbe_get_moments(dvbe_solver s, double *rho, double *ux, double *uy) {
  if (!s || !rho || !ux || !uy) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  const size_t n = (size_t)s->pb.nx * s->pb.ny;
  double *d = (double *)dmalloc(sizeof(double) * 3 * n, s->stream);
  if (!d) return fail(DVBE_ERR_OOM, "device staging allocation failed");
  cudaError_t e = aux_moments(cur_view(s), d, d + n, d + 2 * n, s->stream);
  s->launches += 1;
  double *dst[3] = {rho, ux, uy};
  for (int q = 0; q < 3 && e == cudaSuccess; ++q)
    e = cudaMemcpyAsync(dst[q], d + q * n, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  dfree(d, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "get_moments");
  return DVBE_OK;
}

dvbe_status dvbe_conserved(dvbe_solver s, double out[3]) {
  if (!s || !out) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  double *res = s->red + kReduceBlocks * 3;
  cudaError_t e = aux_conserved(cur_view(s), s->dp.volx, s->dp.voly, s->qvol, s->pb.nx, s->red, res,
                                s->stream);
  s->launches += 2;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "conserved");
  return DVBE_OK;
}

dvbe_status dvbe_residual(dvbe_solver s, double *r) {
  if (!s || !r) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  const size_t n = (size_t)s->pb.nx * s->pb.ny;
  if (!s->uprev) {
    s->uprev = (double *)dmalloc(sizeof(double) * 2 * n, s->stream);
    if (!s->uprev) return fail(DVBE_ERR_OOM, "device allocation failed");
  }
  double *res = s->red + kReduceBlocks * 3;
  cudaError_t e = aux_velocity_error(cur_view(s), s->uprev, s->uprev + n, 1, s->red, res, s->stream);
  s->launches += 2;
  double out[3];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "residual");
  *r = s->have_prev ? std::sqrt(out[0]) / std::sqrt(out[1]) : INFINITY;
  s->have_prev = true;
  return DVBE_OK;
}

dvbe_status dvbe_l2_error_u(dvbe_solver s, const double *ua, const double *va, double *eu) {
  if (!s || !ua || !va || !eu) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  const size_t n = (size_t)s->pb.nx * s->pb.ny;
  const double *src[2] = {ua, va};
  double *d = nullptr;
  dvbe_status st = stage_fields(src, 2, n, s->stream, &d);
  if (st != DVBE_OK) return st;
  double *res = s->red + kReduceBlocks * 3;
  cudaError_t e = aux_velocity_error(cur_view(s), d, d + n, 0, s->red, res, s->stream);
  s->launches += 2;
  double out[3];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  dfree(d, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "l2_error_u");
  *eu = std::sqrt(out[0]) / std::sqrt(out[1]);
  return DVBE_OK;
}

dvbe_status dvbe_get_launch(dvbe_solver s, dvbe_launch *out) {
  if (!s || !out) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  *out = s->launch;
  return DVBE_OK;
}

dvbe_status dvbe_set_launch(dvbe_solver s, const dvbe_launch *in) {
  if (!s || !in) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  if (in->strip_rows < 1 || in->warps_per_block < 1 || in->warps_per_block > 8 || in->blocks < 0 ||
      in->graph_chunk < 0)
    return fail(DVBE_ERR_INVALID_ARG, "strip_rows >= 1, warps_per_block in 1..8, blocks >= 0");
  dvbe_status st = dvbe_sync(s);
  if (st != DVBE_OK && st != DVBE_ERR_DIVERGED) return st;
  s->launch = *in;
  set_strips(s->args, in->strip_rows, s->pb.store);
  drop_graphs(s);
  return DVBE_OK;
}

// Resident blocks per SM of this solver's inner-strip kernel.
static int inner_blocks_per_sm(const Problem &pb, int wpb) {
  switch (pb.store) {
    case ST_F64:
      return inner_blocks_per_sm_f64(pb.kernel, wpb);
    case ST_F32:
    case ST_F32_DEV:
      return inner_blocks_per_sm_f32(pb.store, pb.kernel, wpb);
    default:
      return inner_blocks_per_sm_f16(pb.store, pb.kernel, wpb);
  }
}

// Smallest strip height whose inner strips (set_strips) fit in `waves`
// waves of `slots` resident warps; 0 if the mesh has no inner strips.
static int wave_fitted_rows(const CaseArgs &args, int store, long long slots, int waves) {
  if (slots <= 0) return 0;
  CaseArgs t = args;
  for (int H = 4; H <= t.ny; ++H) {
    set_strips(t, H, store);
    const long long items = (long long)t.in_nx * t.in_ny;
    if (items == 0) return 0;
    if (items <= (long long)waves * slots) return H;
  }
  return 0;
}

static std::string solver_tune_key(dvbe_solver s) {
  char b[160];
  snprintf(b, sizeof b, "k_step|kernel %d|store %d|%dx%d|periodic %d%d", s->pb.kernel, s->pb.store,
           s->pb.nx, s->pb.ny, (int)s->pb.per_x, (int)s->pb.per_y);
  return tune_key(b);
}

static void apply_launch(dvbe_solver s, const dvbe_launch &l) {
  s->launch = l;
  set_strips(s->args, l.strip_rows, s->pb.store);
  drop_graphs(s);
}

dvbe_status dvbe_autotune(dvbe_solver s, int steps, double *best_ms) {
  if (!s || steps < 1) return fail(DVBE_ERR_INVALID_ARG, "bad argument");
  if (s->pb.multipass) { // its kernels take no launch shape
    if (best_ms) *best_ms = 0.0;
    return DVBE_OK;
  }
  const dvbe_launch saved = s->launch;
  const std::string key = solver_tune_key(s);
  TuneEntry hit;
  if (tune_lookup(key, &hit) && hit.strip_rows >= 1 && hit.warps_per_block >= 1 &&
      hit.warps_per_block <= 8 && hit.blocks >= 0) {
    dvbe_status st = dvbe_sync(s);
    if (st != DVBE_OK && st != DVBE_ERR_DIVERGED) return st;
    apply_launch(s, {hit.strip_rows, hit.warps_per_block, hit.blocks, saved.graph_chunk});
    if (best_ms) *best_ms = hit.ms;
    return DVBE_OK;
  }
  const size_t fbytes = (size_t)s->pb.plane * 9 * s->pb.elem;
  void *backup = dmalloc(fbytes, s->stream);
  if (!backup) return fail(DVBE_ERR_OOM, "device allocation failed");
  cudaError_t e = cudaMemcpyAsync(backup, s->f[s->cur], fbytes, cudaMemcpyDeviceToDevice, s->stream);
  const int saved_cur = s->cur;
  const long long saved_steps = s->steps;
  std::vector<dvbe_launch> cand;
  auto add = [&](int H, int w, int blocks) {
    for (auto &c : cand)
      if (c.strip_rows == H && c.warps_per_block == w && c.blocks == blocks) return;
    cand.push_back({H, w, blocks, 0});
  };
  const int rows[] = {8, 16, 24, 32, 48, 64, 128, 256};
  const int wpbs[] = {2, 4, 8};
  for (int w : wpbs) {
    const int wave = inner_blocks_per_sm(s->pb, w) * sm_count(); // blocks in one wave
    std::vector<int> hs;
    for (int H : rows)
      if (H <= 16 || H <= 2 * s->pb.ny) hs.push_back(H);
    for (int k = 1; k <= 3; ++k) {
      const int H = wave_fitted_rows(s->args, s->pb.store, (long long)wave * w, k);
      if (H > 0) hs.push_back(H);
    }
    for (int H : hs) {
      add(H, w, 0);
      if (wave > 0) add(H, w, wave);
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = INFINITY;
  dvbe_launch bestc = saved;
  for (auto &c : cand) {
    if (e != cudaSuccess) break;
    apply_launch(s, c);
    e = launch_one(s); // warm-up
    if (e != cudaSuccess) break;
    cudaEventRecord(e0, s->stream);
    for (int k = 0; k < steps && e == cudaSuccess; ++k) e = launch_one(s);
    cudaEventRecord(e1, s->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms / steps < best) {
      best = ms / steps;
      bestc = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s->cur = saved_cur;
  s->steps = saved_steps;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->f[s->cur], backup, fbytes, cudaMemcpyDeviceToDevice, s->stream);
  unsigned z = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->flag, &z, sizeof z, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  dfree(backup, s->stream);
  bestc.graph_chunk = saved.graph_chunk;
  apply_launch(s, bestc);
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  TuneEntry te;
  te.strip_rows = bestc.strip_rows;
  te.warps_per_block = bestc.warps_per_block;
  te.blocks = bestc.blocks;
  te.ms = best;
  tune_store(key, te);
  if (best_ms) *best_ms = best;
  return DVBE_OK;
}

dvbe_status dvbe_device_state(dvbe_solver s, void **ptr, long long *pitch, long long *plane,
                              int *elem_bytes_) {
  if (!s) return fail(DVBE_ERR_INVALID_ARG, "NULL solver");
  if (ptr) *ptr = cur_view(s).f;
  if (pitch) *pitch = s->pb.pitch;
  if (plane) *plane = s->pb.plane;
  if (elem_bytes_) *elem_bytes_ = s->pb.elem;
  return DVBE_OK;
}

dvbe_status dvbe_launch_count(dvbe_solver s, long long *count) {
  if (!s || !count) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  *count = s->launches;
  return DVBE_OK;
}

static dvbe_status copy_line(dvbe_solver s, int axis, int index, int lo, int hi, void *buf,
                             int to_buf, const char *what) {
  if (!s || !buf) return fail(DVBE_ERR_INVALID_ARG, std::string(what) + ": NULL argument");
  const int nidx = axis == 0 ? s->pb.nx : s->pb.ny, nlen = axis == 0 ? s->pb.ny : s->pb.nx;
  if ((axis != 0 && axis != 1) || index < 0 || index >= nidx || lo < 0 || hi > nlen || lo >= hi)
    return fail(DVBE_ERR_INVALID_ARG, std::string(what) + ": line outside the mesh");
  cudaError_t e = aux_copy_line(cur_view(s), s->pb.elem, axis, index, lo, hi - lo, buf, to_buf, s->stream);
  s->launches += 1;
  if (e == cudaSuccess && !to_buf && s->pb.hx > 0) { // cells may have changed under their copies
    e = aux_fill_halo(cur_view(s), s->pb.hx, s->stream);
    s->launches += 1;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, what);
  return DVBE_OK;
}

dvbe_status dvbe_pack_line(dvbe_solver s, int axis, int index, int lo, int hi, void *dev_buf) {
  return copy_line(s, axis, index, lo, hi, dev_buf, 1, "pack_line");
}

dvbe_status dvbe_unpack_line(dvbe_solver s, int axis, int index, int lo, int hi, const void *dev_buf) {
  return copy_line(s, axis, index, lo, hi, const_cast<void *>(dev_buf), 0, "unpack_line");
}

dvbe_status dvbe_conserved_window(dvbe_solver s, int i0, int j0, int nx, int ny, double out[3]) {
  if (!s || !out) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  if (i0 < 0 || j0 < 0 || nx < 1 || ny < 1 || i0 + nx > s->pb.nx || j0 + ny > s->pb.ny)
    return fail(DVBE_ERR_INVALID_ARG, "window outside the mesh");
  FieldView v = cur_view(s);
  v.f = (char *)v.f + ((long long)j0 * v.pitch + i0) * s->pb.elem;
  v.nx = nx;
  v.ny = ny;
  double *res = s->red + kReduceBlocks * 3;
  cudaError_t e = aux_conserved(v, s->dp.volx + i0, s->dp.voly + j0,
                                s->qvol ? s->qvol + (long long)j0 * s->pb.nx + i0 : nullptr, s->pb.nx,
                                s->red, res, s->stream);
  s->launches += 2;
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "conserved_window");
  return DVBE_OK;
}

dvbe_status dvbe_state_bytes(dvbe_solver s, size_t *bytes) {
  if (!s || !bytes) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  *bytes = (size_t)s->pb.plane * 9 * s->pb.elem;
  return DVBE_OK;
}

dvbe_status dvbe_save_state(dvbe_solver s, void *host, size_t bytes, long long *step) {
  if (!s || !host) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  const size_t fbytes = (size_t)s->pb.plane * 9 * s->pb.elem;
  if (bytes != fbytes)
    return fail(DVBE_ERR_INVALID_ARG, "state buffer must hold " + std::to_string(fbytes) + " bytes");
  cudaError_t e = cudaMemcpyAsync(host, s->f[s->cur], fbytes, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "save_state");
  if (step) *step = s->steps;
  return DVBE_OK;
}

dvbe_status dvbe_load_state(dvbe_solver s, const void *host, size_t bytes, long long step) {
  if (!s || !host || step < 0) return fail(DVBE_ERR_INVALID_ARG, "NULL argument or negative step");
  const size_t fbytes = (size_t)s->pb.plane * 9 * s->pb.elem;
  if (bytes != fbytes)
    return fail(DVBE_ERR_INVALID_ARG, "state buffer must hold " + std::to_string(fbytes) + " bytes");
  cudaError_t e = cudaMemcpyAsync(s->f[s->cur], host, fbytes, cudaMemcpyHostToDevice, s->stream);
  dvbe_status st = after_init(s, e, "load_state");
  if (st != DVBE_OK) return st;
  s->steps = step;
  return DVBE_OK;
}

dvbe_status dvbe_set_wait_limit(dvbe_solver s, long long polls) {
  if (!s || polls < 0) return fail(DVBE_ERR_INVALID_ARG, "NULL solver or negative poll count");
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_wait_limit");
  s->args.wait_limit = (unsigned long long)polls;
  drop_graphs(s); // captured launches hold the old arguments
  return DVBE_OK;
}

} // extern "C"
