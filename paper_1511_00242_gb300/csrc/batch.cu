// Batched form of libdvbe: many independent cases of uneven size advanced
// together.  Each step is one persistent launch per scheme; its warps pull
// strips (strip_cols columns x H rows of one case) from a device work queue that
// covers every case, so small and large meshes share the GPU without a
// launch per case.  Steps are replayed from captured CUDA graphs.  A case
// whose density turns non-finite is flagged and skipped from then on; the
// others are unaffected.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "capi_common.h"

using namespace dvbe;

struct dvbe_batch_ {
  int n = 0, store = 0;
  std::vector<Problem> pb;
  std::vector<DeviceProblem> dp;
  std::vector<CaseArgs> args;
  std::vector<void *> f[2];
  std::vector<CUtensorMap> tm[2][2]; // [buffer parity][main, wrap][case]
  unsigned *flags = nullptr;
  // per buffer parity: case arguments grouped by scheme (DUGKS first), and
  // the strip prefix of each group
  CaseArgs *d_cases[2] = {nullptr, nullptr};
  long long *d_prefix = nullptr; // [2 groups][n+1]
  unsigned long long *d_queue = nullptr;
  std::vector<int> order; // case indices, DUGKS group first
  int ngroup[2] = {0, 0};
  long long nitems[2] = {0, 0};
  cudaStream_t stream = nullptr;
  int cur = 0;
  long long steps = 0, launches = 0;
  dvbe_launch launch{32, 4, 0, 0};
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_len = 0;
};

static void batch_drop_graphs(dvbe_batch b) {
  for (int p = 0; p < 2; ++p)
    if (b->graph[p]) {
      cudaGraphExecDestroy(b->graph[p]);
      b->graph[p] = nullptr;
    }
  b->graph_len = 0;
}

// Rebuild the device case tables for the current strip height.
static dvbe_status batch_tables(dvbe_batch b) {
  std::vector<long long> prefix(2 * (size_t)(b->n + 1), 0);
  for (int g = 0; g < 2; ++g) {
    long long acc = 0;
    const int base = g == 0 ? 0 : b->ngroup[0];
    for (int k = 0; k < b->ngroup[g]; ++k) {
      CaseArgs &a = b->args[b->order[base + k]];
      set_strips(a, b->launch.strip_rows, b->store);
      prefix[g * (size_t)(b->n + 1) + k] = acc;
      acc += (long long)a.strips_x * a.strips_y;
    }
    prefix[g * (size_t)(b->n + 1) + b->ngroup[g]] = acc;
    b->nitems[g] = acc;
  }
  cudaError_t e = cudaSuccess;
  std::vector<CaseArgs> tab(b->n);
  for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
    for (int k = 0; k < b->n; ++k) {
      const int c = b->order[k];
      tab[k] = b->args[c];
      tab[k].tm_main = b->tm[p][0][c];
      tab[k].tm_wrap = b->tm[p][1][c];
      tab[k].fin = b->f[p][c];
      tab[k].fout = b->f[1 - p][c];
      tab[k].flag = b->flags + c;
    }
    e = cudaMemcpyAsync(b->d_cases[p], tab.data(), sizeof(CaseArgs) * b->n, cudaMemcpyHostToDevice,
                        b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_prefix, prefix.data(), sizeof(long long) * prefix.size(),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch tables");
  return DVBE_OK;
}

static cudaError_t batch_launch_one(dvbe_batch b) {
  cudaError_t e = cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(unsigned long long), b->stream);
  const int scheme[2] = {SC_DUGKS, SC_BKG_FV};
  for (int g = 0; g < 2 && e == cudaSuccess; ++g) {
    if (b->ngroup[g] == 0) continue;
    const int base = g == 0 ? 0 : b->ngroup[0];
    e = launch_step_batch(b->store, scheme[g], b->d_cases[b->cur] + base,
                          b->d_prefix + g * (size_t)(b->n + 1), b->ngroup[g], b->nitems[g],
                          b->d_queue + g, b->launch.blocks, b->launch.warps_per_block, b->stream);
    b->launches += 1;
  }
  b->cur ^= 1;
  b->steps += 1;
  return e;
}

extern "C" {

void dvbe_batch_destroy(dvbe_batch b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_drop_graphs(b);
  for (int p = 0; p < 2; ++p) {
    for (void *q : b->f[p]) dfree(q, b->stream);
    dfree(b->d_cases[p], b->stream);
  }
  for (auto &d : b->dp) dfree(d.blob, b->stream);
  dfree(b->flags, b->stream);
  dfree(b->d_prefix, b->stream);
  dfree(b->d_queue, b->stream);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

dvbe_status dvbe_batch_create(const dvbe_params *cases, int ncases, dvbe_batch *out) {
  if (!out || !cases || ncases < 1) return fail(DVBE_ERR_INVALID_ARG, "bad argument");
  *out = nullptr;
  dvbe_batch b = new (std::nothrow) dvbe_batch_;
  if (!b) return fail(DVBE_ERR_OOM, "host allocation failed");
  b->n = ncases;
  b->pb.resize(ncases);
  b->dp.resize(ncases);
  b->args.resize(ncases);
  b->f[0].assign(ncases, nullptr);
  b->f[1].assign(ncases, nullptr);
  for (int p = 0; p < 2; ++p)
    for (int m = 0; m < 2; ++m) b->tm[p][m].resize(ncases);
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "cudaStreamCreate");
  }
  dvbe_status st = DVBE_OK;
  for (int c = 0; c < ncases && st == DVBE_OK; ++c) {
    st = build_problem(&cases[c], b->pb[c], true);
    if (st == DVBE_OK && b->pb[c].kernel == SC_BKG_FD)
      st = fail(DVBE_ERR_UNSUPPORTED, "the batched form runs BKG in finite-volume form only");
    if (st == DVBE_OK && b->pb[c].kernel == SC_CFREE)
      st = fail(DVBE_ERR_UNSUPPORTED, "the batched form runs DUGKS and BKG only");
    if (st == DVBE_OK && b->pb[c].multipass)
      st = fail(DVBE_ERR_UNSUPPORTED, "the batched form runs the fused step with the linear reconstruction");
    if (st == DVBE_OK && c > 0 && b->pb[c].store != b->pb[0].store)
      st = fail(DVBE_ERR_INVALID_ARG, "all cases of a batch must share one precision");
    if (st == DVBE_OK) st = upload_problem(b->pb[c], b->dp[c], b->args[c], b->stream);
    if (st == DVBE_OK) {
      const size_t fbytes = (size_t)b->pb[c].plane * 9 * b->pb[c].elem;
      for (int p = 0; p < 2; ++p) {
        b->f[p][c] = dmalloc(fbytes, b->stream);
        if (!b->f[p][c]) st = fail(DVBE_ERR_OOM, "device allocation of f_tilde failed");
        if (st == DVBE_OK) st = make_tensor_maps(b->pb[c], b->f[p][c], &b->tm[p][0][c], &b->tm[p][1][c]);
      }
    }
    if (st == DVBE_OK) {
      FieldView v = view_of(b->pb[c], b->f[0][c]);
      e = aux_fill_rest(v, b->stream);
      b->launches += 1;
      if (e == cudaSuccess && b->pb[c].hx > 0) {
        e = aux_fill_halo(v, b->pb[c].hx, b->stream);
        b->launches += 1;
      }
      if (e != cudaSuccess) st = cuda_fail(e, "batch initialisation");
    }
  }
  if (st == DVBE_OK) {
    b->store = b->pb[0].store;
    for (int c = 0; c < ncases; ++c)
      if (b->pb[c].user_scheme == DVBE_DUGKS) b->order.push_back(c);
    b->ngroup[0] = (int)b->order.size();
    for (int c = 0; c < ncases; ++c)
      if (b->pb[c].user_scheme != DVBE_DUGKS) b->order.push_back(c);
    b->ngroup[1] = ncases - b->ngroup[0];
    b->flags = (unsigned *)dmalloc(sizeof(unsigned) * ncases, b->stream);
    b->d_cases[0] = (CaseArgs *)dmalloc(sizeof(CaseArgs) * ncases, b->stream);
    b->d_cases[1] = (CaseArgs *)dmalloc(sizeof(CaseArgs) * ncases, b->stream);
    b->d_prefix = (long long *)dmalloc(sizeof(long long) * 2 * (ncases + 1), b->stream);
    b->d_queue = (unsigned long long *)dmalloc(2 * sizeof(unsigned long long), b->stream);
    if (!b->flags || !b->d_cases[0] || !b->d_cases[1] || !b->d_prefix || !b->d_queue)
      st = fail(DVBE_ERR_OOM, "device allocation failed");
  }
  if (st == DVBE_OK) {
    e = cudaMemsetAsync(b->flags, 0, sizeof(unsigned) * ncases, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "batch initialisation");
  }
  if (st == DVBE_OK) st = batch_tables(b);
  if (st != DVBE_OK) {
    dvbe_batch_destroy(b);
    return st;
  }
  *out = b;
  return DVBE_OK;
}

dvbe_status dvbe_batch_init_equilibrium(dvbe_batch b, int c, const double *rho, const double *ux,
                                        const double *uy) {
  if (!b || c < 0 || c >= b->n || !rho || !ux || !uy)
    return fail(DVBE_ERR_INVALID_ARG, "bad argument");
  const size_t n = (size_t)b->pb[c].nx * b->pb[c].ny;
  const double *src[3] = {rho, ux, uy};
  double *d = nullptr;
  dvbe_status st = stage_fields(src, 3, n, b->stream, &d);
  if (st != DVBE_OK) return st;
  cudaError_t e = aux_init_eq(view_of(b->pb[c], b->f[b->cur][c]), d, d + n, d + 2 * n, b->stream);
  b->launches += 1;
  if (e == cudaSuccess && b->pb[c].hx > 0) {
    e = aux_fill_halo(view_of(b->pb[c], b->f[b->cur][c]), b->pb[c].hx, b->stream);
    b->launches += 1;
  }
  unsigned z = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->flags + c, &z, sizeof z, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  dfree(d, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch init_equilibrium");
  return DVBE_OK;
}

static cudaError_t batch_capture(dvbe_batch b, int parity, int len) {
  cudaGraph_t g = nullptr;
  const int saved_cur = b->cur;
  const long long saved_steps = b->steps, saved_l = b->launches;
  b->cur = parity;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < len; ++k) {
    cudaError_t x = batch_launch_one(b);
    if (x != cudaSuccess && le == cudaSuccess) le = x;
  }
  e = cudaStreamEndCapture(b->stream, &g);
  b->cur = saved_cur;
  b->steps = saved_steps;
  b->launches = saved_l;
  if (le != cudaSuccess) e = le;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[parity], g, 0);
  if (g) cudaGraphDestroy(g);
  return e;
}

dvbe_status dvbe_batch_step(dvbe_batch b, long long nsteps, int graph_chunk) {
  if (!b || nsteps < 0 || graph_chunk < 0) return fail(DVBE_ERR_INVALID_ARG, "bad argument");
  cudaError_t e = cudaSuccess;
  int chunk = graph_chunk + (graph_chunk & 1);
  if (chunk > 0 && nsteps >= chunk) {
    if (b->graph_len != chunk) {
      batch_drop_graphs(b);
      for (int p = 0; p < 2 && e == cudaSuccess; ++p) e = batch_capture(b, p, chunk);
      if (e != cudaSuccess) {
        batch_drop_graphs(b);
        return cuda_fail(e, "batch graph capture");
      }
      b->graph_len = chunk;
    }
    const int per_step = (b->ngroup[0] > 0) + (b->ngroup[1] > 0);
    while (nsteps >= chunk && e == cudaSuccess) {
      e = cudaGraphLaunch(b->graph[b->cur], b->stream);
      b->steps += chunk;
      b->launches += (long long)chunk * per_step;
      nsteps -= chunk;
    }
  }
  for (long long k = 0; k < nsteps && e == cudaSuccess; ++k) e = batch_launch_one(b);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch step");
  return DVBE_OK;
}

dvbe_status dvbe_batch_case_status(dvbe_batch b, int c) {
  if (!b || c < 0 || c >= b->n) return fail(DVBE_ERR_INVALID_ARG, "bad argument");
  unsigned flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, b->flags + c, sizeof flag, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch status");
  if (flag & 2u) return fail(DVBE_ERR_TIMEOUT, "a bounded wait in the step kernel ran out");
  if (flag) return fail(DVBE_ERR_DIVERGED, "case diverged");
  return DVBE_OK;
}

dvbe_status dvbe_batch_get_moments(dvbe_batch b, int c, double *rho, double *ux, double *uy) {
  if (!b || c < 0 || c >= b->n || !rho || !ux || !uy)
    return fail(DVBE_ERR_INVALID_ARG, "bad argument");
  const size_t n = (size_t)b->pb[c].nx * b->pb[c].ny;
  double *d = (double *)dmalloc(sizeof(double) * 3 * n, b->stream);
  if (!d) return fail(DVBE_ERR_OOM, "device staging allocation failed");
  cudaError_t e = aux_moments(view_of(b->pb[c], b->f[b->cur][c]), d, d + n, d + 2 * n, b->stream);
  b->launches += 1;
  double *dst[3] = {rho, ux, uy};
  for (int q = 0; q < 3 && e == cudaSuccess; ++q)
    e = cudaMemcpyAsync(dst[q], d + q * n, sizeof(double) * n, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  dfree(d, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch get_moments");
  return DVBE_OK;
}

dvbe_status dvbe_batch_get_f(dvbe_batch b, int c, double *ft) {
  if (!b || c < 0 || c >= b->n || !ft) return fail(DVBE_ERR_INVALID_ARG, "bad argument");
  const size_t n = (size_t)b->pb[c].nx * b->pb[c].ny;
  double *d = (double *)dmalloc(sizeof(double) * n, b->stream);
  if (!d) return fail(DVBE_ERR_OOM, "device staging allocation failed");
  cudaError_t e = cudaSuccess;
  for (int a = 0; a < 9 && e == cudaSuccess; ++a) {
    e = aux_get_field(view_of(b->pb[c], b->f[b->cur][c]), a, d, b->stream);
    b->launches += 1;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ft + a * n, d, sizeof(double) * n, cudaMemcpyDeviceToHost, b->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  dfree(d, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch get_f");
  return DVBE_OK;
}

dvbe_status dvbe_batch_set_launch(dvbe_batch b, const dvbe_launch *in) {
  if (!b || !in) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  if (in->strip_rows < 1 || in->warps_per_block < 1 || in->warps_per_block > 8 || in->blocks < 0)
    return fail(DVBE_ERR_INVALID_ARG, "strip_rows >= 1, warps_per_block in 1..8, blocks >= 0");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch set_launch");
  b->launch = *in;
  batch_drop_graphs(b);
  return batch_tables(b);
}

// Cache key of a batch: storage mode, case count and a hash (FNV-1a) of
// every case's kernel, mesh size and periodicity.
static std::string batch_tune_key(dvbe_batch b) {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](long long v) {
    for (int k = 0; k < 8; ++k) {
      h ^= (unsigned long long)((v >> (8 * k)) & 0xff);
      h *= 1099511628211ull;
    }
  };
  for (int c = 0; c < b->n; ++c) {
    mix(b->pb[c].kernel);
    mix(b->pb[c].nx);
    mix(b->pb[c].ny);
    mix(b->pb[c].per_x * 2 + b->pb[c].per_y);
  }
  char s[160];
  snprintf(s, sizeof s, "k_step_batch|store %d|%d cases|%016llx", b->store, b->n, h);
  return tune_key(s);
}

dvbe_status dvbe_batch_autotune(dvbe_batch b, int steps, double *best_ms) {
  if (!b || steps < 1) return fail(DVBE_ERR_INVALID_ARG, "bad argument");
  const std::string key = batch_tune_key(b);
  TuneEntry hit;
  if (tune_lookup(key, &hit) && hit.strip_rows >= 1 && hit.warps_per_block >= 1 &&
      hit.warps_per_block <= 8 && hit.blocks >= 0) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch autotune");
    b->launch = {hit.strip_rows, hit.warps_per_block, hit.blocks, 0};
    batch_drop_graphs(b);
    if (best_ms) *best_ms = hit.ms;
    return batch_tables(b);
  }
  // back up the current state of every case
  size_t total = 0;
  std::vector<size_t> bytes(b->n);
  for (int c = 0; c < b->n; ++c) {
    bytes[c] = (size_t)b->pb[c].plane * 9 * b->pb[c].elem;
    total += bytes[c];
  }
  char *backup = (char *)dmalloc(total, b->stream);
  if (!backup) return fail(DVBE_ERR_OOM, "device allocation failed");
  cudaError_t e = cudaSuccess;
  size_t pos = 0;
  for (int c = 0; c < b->n && e == cudaSuccess; ++c) {
    e = cudaMemcpyAsync(backup + pos, b->f[b->cur][c], bytes[c], cudaMemcpyDeviceToDevice, b->stream);
    pos += bytes[c];
  }
  unsigned *flags_backup = (unsigned *)dmalloc(sizeof(unsigned) * b->n, b->stream);
  if (!flags_backup) {
    dfree(backup, b->stream);
    return fail(DVBE_ERR_OOM, "device allocation failed");
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(flags_backup, b->flags, sizeof(unsigned) * b->n, cudaMemcpyDeviceToDevice, b->stream);
  const int saved_cur = b->cur;
  const long long saved_steps = b->steps;
  dvbe_launch bestc = b->launch;
  double best = INFINITY;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int rows[] = {8, 16, 32, 64};
  const int wpbs[] = {4, 8};
  for (int H : rows)
    for (int w : wpbs) {
      if (e != cudaSuccess) break;
      b->launch = {H, w, 0, 0};
      dvbe_status st = batch_tables(b);
      if (st != DVBE_OK) {
        e = cudaErrorUnknown;
        break;
      }
      e = batch_launch_one(b);
      cudaEventRecord(e0, b->stream);
      for (int k = 0; k < steps && e == cudaSuccess; ++k) e = batch_launch_one(b);
      cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / steps < best) {
        best = ms / steps;
        bestc = b->launch;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->cur = saved_cur;
  b->steps = saved_steps;
  pos = 0;
  for (int c = 0; c < b->n && e == cudaSuccess; ++c) {
    e = cudaMemcpyAsync(b->f[b->cur][c], backup + pos, bytes[c], cudaMemcpyDeviceToDevice, b->stream);
    pos += bytes[c];
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->flags, flags_backup, sizeof(unsigned) * b->n, cudaMemcpyDeviceToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  dfree(backup, b->stream);
  dfree(flags_backup, b->stream);
  b->launch = bestc;
  batch_drop_graphs(b);
  dvbe_status st = batch_tables(b);
  if (e != cudaSuccess) return cuda_fail(e, "batch autotune");
  if (st != DVBE_OK) return st;
  TuneEntry te;
  te.strip_rows = bestc.strip_rows;
  te.warps_per_block = bestc.warps_per_block;
  te.blocks = bestc.blocks;
  te.ms = best;
  tune_store(key, te);
  if (best_ms) *best_ms = best;
  return DVBE_OK;
}

dvbe_status dvbe_batch_set_wait_limit(dvbe_batch b, long long polls) {
  if (!b || polls < 0) return fail(DVBE_ERR_INVALID_ARG, "NULL batch or negative poll count");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch set_wait_limit");
  for (auto &a : b->args) a.wait_limit = (unsigned long long)polls;
  batch_drop_graphs(b);
  return batch_tables(b);
}

dvbe_status dvbe_batch_launch_count(dvbe_batch b, long long *count) {
  if (!b || !count) return fail(DVBE_ERR_INVALID_ARG, "NULL argument");
  *count = b->launches;
  return DVBE_OK;
}

} // extern "C"
