// FP64 vector kernels for the CG solver: a deterministic two-pass dot product
// (fixed grid, fixed reduction order, so repeated calls give identical bits),
// axpby, pointwise product and reciprocal.  All are HBM-bound streams.
#include "convert.cuh"
#include "mfa_internal.h"

namespace mfa {
namespace {

constexpr int kDotBlocks = 1024;
constexpr int kDotThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kDotThreads) dot_partial_kernel(const double* __restrict__ a,
                                                                  const double* __restrict__ b, int64_t n,
                                                                  double* __restrict__ partial) {
  __shared__ double ws[kDotThreads / 32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kDotThreads)
    s = fma(a[i], b[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kDotThreads / 32 ? ws[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
}

__global__ void __launch_bounds__(kDotThreads) dot_final_kernel(const double* __restrict__ partial,
                                                                double* __restrict__ out) {
  __shared__ double ws[kDotThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += kDotThreads) s += partial[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kDotThreads / 32 ? ws[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *out = v;
  }
}

__global__ void axpby_kernel(double alpha, const double* __restrict__ x, double beta, double* __restrict__ y,
                             int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = alpha * x[i] + beta * y[i];
}

__global__ void mul_kernel(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                           int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] * b[i];
}

// Dirichlet constraints: mask[i] != 0 marks a constrained dof.
__global__ void dir_mask_kernel(const double* __restrict__ x, const uint8_t* __restrict__ mask,
                                double* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = mask[i] ? 0.0 : x[i];
}

__global__ void dir_combine_kernel(const double* __restrict__ ax, const double* __restrict__ x,
                                   const uint8_t* __restrict__ mask, double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += mask[i] ? x[i] : ax[i];
}

__global__ void dir_diag_kernel(const uint8_t* __restrict__ mask, double* __restrict__ d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (mask[i]) d[i] = 1.0;
}

__global__ void recip_kernel(const double* __restrict__ a, double* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = 1.0 / a[i];
}

// y += sign * (num / den) * x with the scalars read on the device.
__global__ void axpy_ratio_kernel(const double* __restrict__ x, double* __restrict__ y, int64_t n,
                                  const double* __restrict__ num, const double* __restrict__ den, double sign) {
  const double a = sign * (*num / *den);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

// p = z + (num / den) * p
__global__ void xpby_ratio_kernel(const double* __restrict__ z, double* __restrict__ p, int64_t n,
                                  const double* __restrict__ num, const double* __restrict__ den) {
  const double beta = *num / *den;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

__global__ void d2f_kernel(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = d2f_bits(x[i]);
}

__global__ void f2d_kernel(const float* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = f2d_bits(x[i]);
}

// ---- float-vector kernels of the inner (reduced-precision) Krylov loop.
// Per-thread sums in float over a few dozen entries, then double across the
// block and across blocks (dot_final_kernel): deterministic for a fixed grid.

__device__ __forceinline__ void block_partial(double v, double* partial) {
  __shared__ double ws[kDotThreads / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < kDotThreads / 32 ? ws[threadIdx.x] : 0.0;
    w = warp_sum(w);
    if (threadIdx.x == 0) partial[blockIdx.x] = w;
  }
}

__global__ void __launch_bounds__(kDotThreads) dot32_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                                            int64_t n, double* __restrict__ partial) {
  float s = 0.0f;
  for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kDotThreads)
    s = fmaf(a[i], b[i], s);
  block_partial(f2d_bits(s), partial);
}

// z = d * r, p = z, partial sums of r . z
__global__ void __launch_bounds__(kDotThreads) jacobi_init32_kernel(const float* __restrict__ d,
                                                                    const float* __restrict__ r, float* __restrict__ z,
                                                                    float* __restrict__ p, int64_t n,
                                                                    double* __restrict__ partial) {
  float s = 0.0f;
  for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kDotThreads) {
    const float zi = d[i] * r[i];
    z[i] = zi;
    p[i] = zi;
    s = fmaf(r[i], zi, s);
  }
  block_partial(f2d_bits(s), partial);
}

// alpha = rz / pq; x += alpha p; r -= alpha q; z = d * r; partial sums of r . z
__global__ void __launch_bounds__(kDotThreads) cg_update32_kernel(const float* __restrict__ p,
                                                                  const float* __restrict__ q, float* __restrict__ r,
                                                                  float* __restrict__ x, const float* __restrict__ d,
                                                                  float* __restrict__ z, int64_t n,
                                                                  const double* __restrict__ rz,
                                                                  const double* __restrict__ pq,
                                                                  double* __restrict__ partial) {
  const float alpha = d2f_bits(*rz / *pq);
  float s = 0.0f;
  for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kDotThreads) {
    x[i] = fmaf(alpha, p[i], x[i]);
    const float ri = fmaf(-alpha, q[i], r[i]);
    r[i] = ri;
    const float zi = d[i] * ri;
    z[i] = zi;
    s = fmaf(ri, zi, s);
  }
  block_partial(f2d_bits(s), partial);
}

// p = z + (num / den) p
__global__ void xpby32_kernel(const float* __restrict__ z, float* __restrict__ p, int64_t n,
                              const double* __restrict__ num, const double* __restrict__ den) {
  const float beta = d2f_bits(*num / *den);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fmaf(beta, p[i], z[i]);
}

// y += sign * (num / den) * x  (float vectors, device scalars)
__global__ void axpy32_ratio_kernel(const float* __restrict__ x, float* __restrict__ y, int64_t n,
                                    const double* __restrict__ num, const double* __restrict__ den, float sign) {
  const float a = sign * d2f_bits(*num / *den);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fmaf(a, x[i], y[i]);
}

// p = z + sign * (num / den) * p
__global__ void xpay32_ratio_kernel(const float* __restrict__ z, float* __restrict__ p, int64_t n,
                                    const double* __restrict__ num, const double* __restrict__ den, float sign) {
  const float beta = sign * d2f_bits(*num / *den);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fmaf(beta, p[i], z[i]);
}

unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

int dot_partials() { return kDotBlocks; }

cudaError_t dot_launch(const double* a, const double* b, int64_t n, double* partial, double* out, cudaStream_t s) {
  dot_partial_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(a, b, n, partial);
  dot_final_kernel<<<1, kDotThreads, 0, s>>>(partial, out);
  return cudaGetLastError();
}

cudaError_t axpby_launch(double alpha, const double* x, double beta, double* y, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  axpby_kernel<<<grid_for(n), 256, 0, s>>>(alpha, x, beta, y, n);
  return cudaGetLastError();
}

cudaError_t dirichlet_mask_launch(const double* x, const uint8_t* mask, double* out, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  dir_mask_kernel<<<grid_for(n), 256, 0, s>>>(x, mask, out, n);
  return cudaGetLastError();
}

cudaError_t dirichlet_combine_launch(const double* ax, const double* x, const uint8_t* mask, double* y, int64_t n,
                                     cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  dir_combine_kernel<<<grid_for(n), 256, 0, s>>>(ax, x, mask, y, n);
  return cudaGetLastError();
}

cudaError_t dirichlet_diag_launch(const uint8_t* mask, double* d, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  dir_diag_kernel<<<grid_for(n), 256, 0, s>>>(mask, d, n);
  return cudaGetLastError();
}

cudaError_t pointwise_mul_launch(const double* a, const double* b, double* out, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  mul_kernel<<<grid_for(n), 256, 0, s>>>(a, b, out, n);
  return cudaGetLastError();
}

cudaError_t axpy_ratio_launch(const double* x, double* y, int64_t n, const double* num, const double* den, double sign,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  axpy_ratio_kernel<<<grid_for(n), 256, 0, s>>>(x, y, n, num, den, sign);
  return cudaGetLastError();
}

cudaError_t xpby_ratio_launch(const double* z, double* p, int64_t n, const double* num, const double* den,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  xpby_ratio_kernel<<<grid_for(n), 256, 0, s>>>(z, p, n, num, den);
  return cudaGetLastError();
}

cudaError_t convert_d2f_launch(const double* x, float* y, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  d2f_kernel<<<grid_for(n), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t convert_f2d_launch(const float* x, double* y, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  f2d_kernel<<<grid_for(n), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t dot32_launch(const float* a, const float* b, int64_t n, double* partial, double* out, cudaStream_t s) {
  dot32_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(a, b, n, partial);
  dot_final_kernel<<<1, kDotThreads, 0, s>>>(partial, out);
  return cudaGetLastError();
}

cudaError_t jacobi_init32_launch(const float* d, const float* r, float* z, float* p, int64_t n, double* partial,
                                 double* out, cudaStream_t s) {
  jacobi_init32_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(d, r, z, p, n, partial);
  dot_final_kernel<<<1, kDotThreads, 0, s>>>(partial, out);
  return cudaGetLastError();
}

cudaError_t cg_update32_launch(const float* p, const float* q, float* r, float* x, const float* d, float* z,
                               int64_t n, const double* rz, const double* pq, double* partial, double* rz_new,
                               cudaStream_t s) {
  cg_update32_kernel<<<kDotBlocks, kDotThreads, 0, s>>>(p, q, r, x, d, z, n, rz, pq, partial);
  dot_final_kernel<<<1, kDotThreads, 0, s>>>(partial, rz_new);
  return cudaGetLastError();
}

cudaError_t xpby32_launch(const float* z, float* p, int64_t n, const double* num, const double* den, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  xpby32_kernel<<<grid_for(n), 256, 0, s>>>(z, p, n, num, den);
  return cudaGetLastError();
}

cudaError_t axpy32_ratio_launch(const float* x, float* y, int64_t n, const double* num, const double* den, float sign,
                                cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  axpy32_ratio_kernel<<<grid_for(n), 256, 0, s>>>(x, y, n, num, den, sign);
  return cudaGetLastError();
}

cudaError_t xpay32_ratio_launch(const float* z, float* p, int64_t n, const double* num, const double* den, float sign,
                                cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  xpay32_ratio_kernel<<<grid_for(n), 256, 0, s>>>(z, p, n, num, den, sign);
  return cudaGetLastError();
}

cudaError_t reciprocal_launch(const double* a, double* out, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  recip_kernel<<<grid_for(n), 256, 0, s>>>(a, out, n);
  return cudaGetLastError();
}

}  // namespace mfa
