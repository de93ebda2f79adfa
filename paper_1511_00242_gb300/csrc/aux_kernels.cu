// Initialisation, codec, moments and FP64 reduction kernels of libdvbe.
//
// All of these run in FP64 regardless of the storage mode: they convert
// between the caller's float64 arrays and the device storage of f_tilde, and
// reduce conserved quantities and error norms in a fixed order (the grid size
// is fixed and every block sums its cells sequentially, then as a tree), so
// results are bitwise reproducible from run to run.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace dvbe {
namespace {

__host__ __device__ constexpr int AEX(int a) {
  return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__host__ __device__ constexpr int AEY(int a) {
  return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}
__host__ __device__ constexpr double AW(int a) {
  return a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

__host__ __device__ constexpr int AWC(int a) { return a == 0 ? 0 : (a <= 4 ? 1 : 2); }

// Read / write f_tilde_alpha of one cell in any storage mode, in FP64.
__device__ __forceinline__ double rd(const FieldView &v, int a, long long idx) {
  const double base = AW(a) * v.rho0, sc = v.scale[AWC(a)];
  switch (v.store) {
    case ST_F64:
      return ((const double *)v.f)[a * v.plane + idx];
    case ST_F32:
      return (double)((const float *)v.f)[a * v.plane + idx];
    case ST_F32_DEV:
      return base + sc * (double)((const float *)v.f)[a * v.plane + idx];
    case ST_F16_DEV:
      return base + sc * (double)__half2float(((const __half *)v.f)[a * v.plane + idx]);
    default:
      return base + sc * (double)__bfloat162float(((const __nv_bfloat16 *)v.f)[a * v.plane + idx]);
  }
}

__device__ __forceinline__ void wr(const FieldView &v, int a, long long idx, double x) {
  const double base = AW(a) * v.rho0;
  const double d = (x - base) / v.scale[AWC(a)];
  switch (v.store) {
    case ST_F64:
      ((double *)v.f)[a * v.plane + idx] = x;
      break;
    case ST_F32:
      ((float *)v.f)[a * v.plane + idx] = (float)x;
      break;
    case ST_F32_DEV:
      ((float *)v.f)[a * v.plane + idx] = (float)d;
      break;
    case ST_F16_DEV:
      ((__half *)v.f)[a * v.plane + idx] = __double2half(d);
      break;
    default:
      ((__nv_bfloat16 *)v.f)[a * v.plane + idx] = __double2bfloat16(d);
      break;
  }
}

__device__ __forceinline__ void feq9(double RT, double rho, double ux, double uy, double *f) {
  const double c = sqrt(3.0 * RT), cs2 = RT;
  const double usq = ux * ux + uy * uy;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    double eu = c * (AEX(a) * ux + AEY(a) * uy);
    f[a] = AW(a) * rho * (1.0 + eu / cs2 + eu * eu / (2.0 * cs2 * cs2) - usq / (2.0 * cs2));
  }
}

__device__ __forceinline__ void mom9(double RT, const double *f, double &rho, double &ux,
                                     double &uy) {
  const double c = sqrt(3.0 * RT);
  double r = 0, jx = 0, jy = 0;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    r += f[a];
    jx += AEX(a) * f[a];
    jy += AEY(a) * f[a];
  }
  rho = r;
  ux = c * jx / r;
  uy = c * jy / r;
}

__global__ void k_init_eq(FieldView v, const double *rho, const double *ux, const double *uy) {
  const long long n = (long long)v.nx * v.ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(k / v.nx), i = (int)(k % v.nx);
    double f[9];
    feq9(v.RT, rho[k], ux[k], uy[k], f);
    const long long idx = (long long)j * v.pitch + i;
#pragma unroll
    for (int a = 0; a < 9; ++a) wr(v, a, idx, f[a]);
  }
}

// Sec 3.1: f = f_eq - tau (d_t f_eq + xi . grad f_eq) through (rho, u), then
// f_tilde = f - dt/2 (f_eq(f) - f)/tau with f_eq of f's own moments.
__global__ void k_init_ce(FieldView v, const double *rho, const double *ux, const double *uy,
                          const double *d0, const double *d1, const double *d2, const double *d3,
                          const double *d4, const double *d5, const double *d6, const double *d7,
                          const double *d8) {
  const long long n = (long long)v.nx * v.ny;
  const double c = sqrt(3.0 * v.RT), cs2 = v.RT;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(k / v.nx), i = (int)(k % v.nx);
    const double r = rho[k], u = ux[k], w = uy[k];
    double fe[9], f[9];
    feq9(v.RT, r, u, w, fe);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const double cx = c * AEX(a), cy = c * AEY(a);
      const double eu = cx * u + cy * w;
      const double dr = fe[a] / r;
      const double du = AW(a) * r * (cx / cs2 + eu * cx / (cs2 * cs2) - u / cs2);
      const double dv = AW(a) * r * (cy / cs2 + eu * cy / (cs2 * cs2) - w / cs2);
      const double ft = dr * d0[k] + du * d1[k] + dv * d2[k];
      const double fx = dr * d3[k] + du * d4[k] + dv * d5[k];
      const double fy = dr * d6[k] + du * d7[k] + dv * d8[k];
      f[a] = fe[a] - v.tau * (ft + cx * fx + cy * fy);
    }
    double rr, uu, vv, g[9];
    mom9(v.RT, f, rr, uu, vv);
    feq9(v.RT, rr, uu, vv, g);
    const long long idx = (long long)j * v.pitch + i;
#pragma unroll
    for (int a = 0; a < 9; ++a) wr(v, a, idx, f[a] - 0.5 * v.dt * (g[a] - f[a]) / v.tau);
  }
}

__global__ void k_fill_rest(FieldView v) {
  const long long n = (long long)v.nx * v.ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(k / v.nx), i = (int)(k % v.nx);
    const long long idx = (long long)j * v.pitch + i;
#pragma unroll
    for (int a = 0; a < 9; ++a) wr(v, a, idx, AW(a) * v.rho0);
  }
}

__global__ void k_set_field(FieldView v, int a, const double *src) {
  const long long n = (long long)v.nx * v.ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(k / v.nx), i = (int)(k % v.nx);
    wr(v, a, (long long)j * v.pitch + i, src[k]);
  }
}

__global__ void k_get_field(FieldView v, int a, double *dst) {
  const long long n = (long long)v.nx * v.ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(k / v.nx), i = (int)(k % v.nx);
    dst[k] = rd(v, a, (long long)j * v.pitch + i);
  }
}

__device__ __forceinline__ void cell_moments(const FieldView &v, long long k, double &rho,
                                             double &ux, double &uy) {
  const int j = (int)(k / v.nx), i = (int)(k % v.nx);
  const long long idx = (long long)j * v.pitch + i;
  double f[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) f[a] = rd(v, a, idx);
  mom9(v.RT, f, rho, ux, uy);
}

__global__ void k_moments(FieldView v, double *rho, double *ux, double *uy) {
  const long long n = (long long)v.nx * v.ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    double r, u, w;
    cell_moments(v, k, r, u, w);
    rho[k] = r;
    ux[k] = u;
    uy[k] = w;
  }
}

constexpr int kRT = 256; // reduction threads per block

// Block tree reduction of 3 sums; thread 0 writes partials[blockIdx.x*3 + q].
__device__ __forceinline__ void block_reduce3(double s0, double s1, double s2, double *partials) {
  __shared__ double sh[3][kRT];
  sh[0][threadIdx.x] = s0;
  sh[1][threadIdx.x] = s1;
  sh[2][threadIdx.x] = s2;
  __syncthreads();
  for (int w = kRT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) partials[blockIdx.x * 3 + q] = sh[q][0];
  }
}

__global__ void k_conserved(FieldView v, const double *volx, const double *voly, const double *volc,
                            long long vpitch, double *partials) {
  const long long n = (long long)v.nx * v.ny;
  double m = 0, jx = 0, jy = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(k / v.nx), i = (int)(k % v.nx);
    double r, u, w;
    cell_moments(v, k, r, u, w);
    const double vol = volc ? volc[(long long)j * vpitch + i] : volx[i] * voly[j];
    m += r * vol;
    jx += r * u * vol;
    jy += r * w * vol;
  }
  block_reduce3(m, jx, jy, partials);
}

__global__ void k_velocity_error(FieldView v, double *ua, double *va, int mode, double *partials) {
  const long long n = (long long)v.nx * v.ny;
  double num = 0, den = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    double r, u, w;
    cell_moments(v, k, r, u, w);
    const double du = u - ua[k], dv = w - va[k];
    num += du * du + dv * dv;
    if (mode == 0) {
      den += ua[k] * ua[k] + va[k] * va[k];
    } else {
      den += u * u + w * w;
      ua[k] = u;
      va[k] = w;
    }
  }
  block_reduce3(num, den, 0.0, partials);
}

__global__ void k_finish3(const double *partials, int nblocks, double *out) {
  // single thread, fixed order
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s[3] = {0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
      for (int q = 0; q < 3; ++q) s[q] += partials[b * 3 + q];
    for (int q = 0; q < 3; ++q) out[q] = s[q];
  }
}

// One line of cells of all nine fields copied between the f_tilde storage
// and a dense buffer [9][n] of the same element type (es bytes): axis 0 is
// column `index` over rows lo .. lo+n-1, axis 1 row `index` over columns
// lo .. lo+n-1; to_buf selects the direction.  Values are moved as stored.
__global__ void k_copy_line(FieldView v, int es, int axis, int index, int lo, int n, char *buf,
                            int to_buf) {
  const long long total = 9LL * n;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(k / n), p = lo + (int)(k % n);
    const long long idx = axis == 0 ? (long long)p * v.pitch + index : (long long)index * v.pitch + p;
    char *cell = (char *)v.f + (a * v.plane + idx) * es;
    char *b = buf + k * es;
    char *dst = to_buf ? b : cell;
    const char *src = to_buf ? cell : b;
    if (es == 8)
      *(unsigned long long *)dst = *(const unsigned long long *)src;
    else if (es == 4)
      *(unsigned *)dst = *(const unsigned *)src;
    else
      *(unsigned short *)dst = *(const unsigned short *)src;
  }
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

} // namespace

cudaError_t aux_init_eq(const FieldView &v, const double *r, const double *u, const double *w,
                        cudaStream_t s) {
  k_init_eq<<<grid_for((long long)v.nx * v.ny), 256, 0, s>>>(v, r, u, w);
  return cudaGetLastError();
}

cudaError_t aux_init_ce(const FieldView &v, const double *r, const double *u, const double *w,
                        const double *const *d, cudaStream_t s) {
  k_init_ce<<<grid_for((long long)v.nx * v.ny), 256, 0, s>>>(v, r, u, w, d[0], d[1], d[2], d[3],
                                                              d[4], d[5], d[6], d[7], d[8]);
  return cudaGetLastError();
}

cudaError_t aux_fill_rest(const FieldView &v, cudaStream_t s) {
  k_fill_rest<<<grid_for((long long)v.nx * v.ny), 256, 0, s>>>(v);
  return cudaGetLastError();
}

template <typename E> __global__ void k_fill_halo(FieldView v, int hx) {
  const long long n = 9LL * v.ny * 2 * hx;
  E *f = (E *)v.f;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t % (2 * hx));
    const long long r = t / (2 * hx);
    const int j = (int)(r % v.ny), a = (int)(r / v.ny);
    E *row = f + (long long)a * v.plane + (long long)j * v.pitch;
    if (q < hx)
      row[q - hx] = row[v.nx - hx + q];
    else
      row[v.nx + (q - hx)] = row[q - hx];
  }
}

cudaError_t aux_fill_halo(const FieldView &v, int hx, cudaStream_t s) {
  const long long n = 9LL * v.ny * 2 * hx;
  if (v.store == ST_F64)
    k_fill_halo<double><<<grid_for(n), 256, 0, s>>>(v, hx);
  else if (v.store == ST_F16_DEV || v.store == ST_BF16_DEV)
    k_fill_halo<unsigned short><<<grid_for(n), 256, 0, s>>>(v, hx);
  else
    k_fill_halo<float><<<grid_for(n), 256, 0, s>>>(v, hx);
  return cudaGetLastError();
}

cudaError_t aux_set_field(const FieldView &v, int a, const double *src, cudaStream_t s) {
  k_set_field<<<grid_for((long long)v.nx * v.ny), 256, 0, s>>>(v, a, src);
  return cudaGetLastError();
}

cudaError_t aux_get_field(const FieldView &v, int a, double *dst, cudaStream_t s) {
  k_get_field<<<grid_for((long long)v.nx * v.ny), 256, 0, s>>>(v, a, dst);
  return cudaGetLastError();
}

cudaError_t aux_moments(const FieldView &v, double *r, double *u, double *w, cudaStream_t s) {
  k_moments<<<grid_for((long long)v.nx * v.ny), 256, 0, s>>>(v, r, u, w);
  return cudaGetLastError();
}

cudaError_t aux_conserved(const FieldView &v, const double *volx, const double *voly,
                          const double *volc, long long vpitch, double *partials, double *out,
                          cudaStream_t s) {
  k_conserved<<<kReduceBlocks, kRT, 0, s>>>(v, volx, voly, volc, vpitch, partials);
  k_finish3<<<1, 32, 0, s>>>(partials, kReduceBlocks, out);
  return cudaGetLastError();
}

cudaError_t aux_copy_line(const FieldView &v, int elem, int axis, int index, int lo, int n,
                          void *buf, int to_buf, cudaStream_t s) {
  k_copy_line<<<grid_for(9LL * n), 256, 0, s>>>(v, elem, axis, index, lo, n, (char *)buf, to_buf);
  return cudaGetLastError();
}

cudaError_t aux_velocity_error(const FieldView &v, double *ua, double *va, int mode,
                               double *partials, double *out, cudaStream_t s) {
  k_velocity_error<<<kReduceBlocks, kRT, 0, s>>>(v, ua, va, mode, partials);
  k_finish3<<<1, 32, 0, s>>>(partials, kReduceBlocks, out);
  return cudaGetLastError();
}

} // namespace dvbe
