// dvbe_conserved_noalloc: the FP64 mass / momentum sums of dvbe_conserved for
// callers that cannot allocate device memory.
//
// Some callers own every byte of device memory they use and cannot let a
// library allocate behind their back: a framework that reserves the GPU's
// memory for its own pool up front, or a time-critical loop where
// cudaMalloc / cudaFree must not run because cudaFree waits for the whole
// device.  This entry point works on buffers the caller already holds
// (f_tilde, the cell widths, a 3-double result) and keeps its partial sums in
// a fixed file-scope device array instead of allocating them.
//
// The scratch array is kNoAllocBlocks x 3 doubles (192 KB), resident on every
// GPU that loads the library until the process exits.  Each reduction block
// handles kNoAllocCellsPerBlock cells, so a mesh may have at most
// kNoAllocBlocks * kNoAllocCellsPerBlock = 33,554,432 cells (8192 x 4096);
// larger meshes are rejected with DVBE_ERR_INVALID_ARG.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>
#include <string>

#include "capi_common.h"

namespace {

constexpr int kNoAllocBlocks = 8192;
constexpr int kNoAllocThreads = 256;
constexpr long long kNoAllocCellsPerBlock = 4096;

// Partial sums of the reduction, shared by every call on a device.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocBlocks * 3];

// Device address of the array, resolved once per device (host code cannot
// use the symbol itself as a device pointer).
constexpr int kMaxDevices = 64;
double *g_scratch[kMaxDevices] = {};
std::mutex g_scratch_mu;

__host__ __device__ constexpr int NEX(int a) {
  return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__host__ __device__ constexpr int NEY(int a) {
  return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}
__host__ __device__ constexpr double NW(int a) {
  return a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

struct View {
  const void *f;
  long long pitch, plane;
  int nx, ny, store;
  double rho0, scale[3], c;
};

__device__ __forceinline__ double value(const View &v, int a, long long idx) {
  const double base = NW(a) * v.rho0, sc = v.scale[a == 0 ? 0 : (a <= 4 ? 1 : 2)];
  switch (v.store) {
    case DVBE_F64:
      return ((const double *)v.f)[a * v.plane + idx];
    case DVBE_F32:
      return (double)((const float *)v.f)[a * v.plane + idx];
    case DVBE_F32_DEV:
      return base + sc * (double)((const float *)v.f)[a * v.plane + idx];
    case DVBE_F16_DEV:
      return base + sc * (double)__half2float(((const __half *)v.f)[a * v.plane + idx]);
    default:
      return base + sc * (double)__bfloat162float(((const __nv_bfloat16 *)v.f)[a * v.plane + idx]);
  }
}

// Pass 1: block b sums cells [b * kNoAllocCellsPerBlock, (b+1) * ...) in a
// fixed order (thread-strided, then a tree) into partials[3b .. 3b+2].
__global__ void k_noalloc_sums(View v, const double *dx, const double *dy, double *partials) {
  __shared__ double sh[3][kNoAllocThreads];
  const long long n = (long long)v.nx * v.ny;
  const long long k0 = (long long)blockIdx.x * kNoAllocCellsPerBlock;
  const long long k1 = k0 + kNoAllocCellsPerBlock < n ? k0 + kNoAllocCellsPerBlock : n;
  double m = 0, jx = 0, jy = 0;
  for (long long k = k0 + threadIdx.x; k < k1; k += kNoAllocThreads) {
    const int j = (int)(k / v.nx), i = (int)(k % v.nx);
    const long long idx = (long long)j * v.pitch + i;
    double r = 0, mx = 0, my = 0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const double fa = value(v, a, idx);
      r += fa;
      mx += NEX(a) * fa;
      my += NEY(a) * fa;
    }
    const double vol = dx[i] * dy[j];
    m += r * vol;
    jx += v.c * mx * vol;
    jy += v.c * my * vol;
  }
  sh[0][threadIdx.x] = m;
  sh[1][threadIdx.x] = jx;
  sh[2][threadIdx.x] = jy;
  __syncthreads();
  for (int w = kNoAllocThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) partials[3 * blockIdx.x + q] = sh[q][0];
}

// Pass 2: one thread adds the nblocks partials in order.
__global__ void k_noalloc_finish(const double *partials, int nblocks, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s[3] = {0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
      for (int q = 0; q < 3; ++q) s[q] += partials[3 * b + q];
    for (int q = 0; q < 3; ++q) out[q] = s[q];
  }
}

// Address of the scratch array on the current device; resolved on the first
// call per device and cached.
dvbe_status scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return dvbe::cuda_fail(e, "dvbe_conserved_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return dvbe::fail(DVBE_ERR_UNSUPPORTED, "dvbe_conserved_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess)
      return dvbe::cuda_fail(e, "dvbe_conserved_noalloc: cudaGetSymbolAddress of the scratch array");
    g_scratch[dev] = (double *)p;
  }
  *out = g_scratch[dev];
  return DVBE_OK;
}

} // namespace

extern "C" DVBE_API dvbe_status dvbe_conserved_noalloc(const void *f_tilde, int precision, int nx,
                                                      int ny, long long pitch, const double *dx,
                                                      const double *dy, double RT, double rho0,
                                                      double dev_scale, double *out, void *stream) {
  if (!f_tilde || !dx || !dy || !out)
    return dvbe::fail(DVBE_ERR_INVALID_ARG, "dvbe_conserved_noalloc: NULL pointer");
  if (nx < 1 || ny < 1 || pitch < nx || !(RT > 0))
    return dvbe::fail(DVBE_ERR_INVALID_ARG, "dvbe_conserved_noalloc: bad size or RT");
  if (precision < DVBE_F64 || precision > DVBE_BF16_DEV)
    return dvbe::fail(DVBE_ERR_INVALID_ARG, "dvbe_conserved_noalloc: unknown precision");
  const long long n = (long long)nx * ny;
  const long long nblocks = (n + kNoAllocCellsPerBlock - 1) / kNoAllocCellsPerBlock;
  if (nblocks > kNoAllocBlocks)
    return dvbe::fail(DVBE_ERR_INVALID_ARG,
                      "dvbe_conserved_noalloc: mesh has " + std::to_string(n) +
                          " cells, more than the " +
                          std::to_string((long long)kNoAllocBlocks * kNoAllocCellsPerBlock) +
                          " its fixed scratch array covers");
  double *scratch = nullptr;
  dvbe_status st = scratch_for_current_device(&scratch);
  if (st != DVBE_OK) return st;
  View v;
  v.f = f_tilde;
  v.pitch = pitch;
  v.plane = pitch * ny;
  v.nx = nx;
  v.ny = ny;
  v.store = precision;
  v.rho0 = rho0 > 0 ? rho0 : 1.0;
  dvbe::deviation_scales(precision, dev_scale, v.rho0, v.scale);
  v.c = sqrt(3.0 * RT);
  cudaStream_t s = (cudaStream_t)stream;
  k_noalloc_sums<<<(int)nblocks, kNoAllocThreads, 0, s>>>(v, dx, dy, scratch);
  k_noalloc_finish<<<1, 32, 0, s>>>(scratch, (int)nblocks, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dvbe::cuda_fail(e, "dvbe_conserved_noalloc: launch");
  return DVBE_OK;
}
