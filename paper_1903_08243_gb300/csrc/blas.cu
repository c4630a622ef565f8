// FP64 vector kernels for the CG solver: a deterministic two-pass dot product
// (fixed grid, fixed reduction order, so repeated calls give identical bits),
// axpby, pointwise product and reciprocal.  All are HBM-bound streams.
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

cudaError_t reciprocal_launch(const double* a, double* out, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  recip_kernel<<<grid_for(n), 256, 0, s>>>(a, out, n);
  return cudaGetLastError();
}

}  // namespace mfa
