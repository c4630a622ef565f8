// FP64 FMA throughput probe: the measured denominator of the FP64 rooflines.
//
// Every FP64 operator of this library is bound by the FP64 pipe (its
// arithmetic intensity is far above the FP64 ridge point), so its roofline
// fraction divides by the rate at which the GPU retires FP64 FMAs.  This
// kernel keeps that pipe busy with nothing else: every thread runs eight
// independent FMA chains (enough to cover the pipe's latency), one wave of
// blocks fills every SM, and each block reads the SM clock and the global
// timer at its start and end, so that the clock under load is measured too.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "mfa_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(kThreads) fp64_fma_probe_kernel(int iters, double* sink, long long* stamps) {
  const long long c0 = clock64();
  const unsigned long long t0 = global_ns();
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  const double m = 0.9999999, c = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == 12345.678) sink[0] = s;  // never true; keeps the chains alive
  __syncthreads();
  if (threadIdx.x == 0) {
    stamps[4 * blockIdx.x + 0] = c0;
    stamps[4 * blockIdx.x + 1] = clock64();
    stamps[4 * blockIdx.x + 2] = (long long)t0;
    stamps[4 * blockIdx.x + 3] = (long long)global_ns();
  }
}

}  // namespace

extern "C" int mfa_probe_fp64_fma(mfa_ctx* ctx, double* tflops, double* sm_mhz) {
  if (!ctx || !tflops) return mfa::set_error(MFA_ERR_ARG, "mfa_probe_fp64_fma: NULL argument");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return mfa::set_error(MFA_ERR_CUDA, "mfa_probe_fp64_fma: device");
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fp64_fma_probe_kernel, kThreads, 0) != cudaSuccess ||
      bps < 1)
    bps = 1;
  const int blocks = ctx->sm_count * bps;  // one full wave
  const int iters = 1 << 15;
  double* sink = nullptr;
  long long* stamps = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int rc = MFA_OK;
  float ms = 0.0f;
  std::vector<long long> h(4 * (size_t)blocks);
  if (cudaMalloc((void**)&sink, sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&stamps, sizeof(long long) * h.size()) != cudaSuccess) {
    rc = mfa::set_error(MFA_ERR_OOM, "mfa_probe_fp64_fma: device allocation");
  } else if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
    rc = mfa::set_error(MFA_ERR_CUDA, "mfa_probe_fp64_fma: events");
  } else {
    mfa::clear_stale_error();
    fp64_fma_probe_kernel<<<blocks, kThreads, 0, ctx->stream>>>(iters / 8, sink, stamps);  // warm-up
    cudaEventRecord(ev[0], ctx->stream);
    fp64_fma_probe_kernel<<<blocks, kThreads, 0, ctx->stream>>>(iters, sink, stamps);
    cudaEventRecord(ev[1], ctx->stream);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (e == cudaSuccess)
      e = cudaMemcpy(h.data(), stamps, sizeof(long long) * h.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = mfa::set_error(MFA_ERR_CUDA, cudaGetErrorString(e));
  }
  if (rc == MFA_OK) {
    const double flops = 2.0 * kChains * (double)iters * kThreads * blocks;
    *tflops = flops / (ms * 1e-3) / 1e12;
    if (sm_mhz) {  // median over blocks of SM clocks per nanosecond
      std::vector<double> mhz;
      for (int b = 0; b < blocks; ++b) {
        const double dns = (double)(h[4 * b + 3] - h[4 * b + 2]);
        if (dns > 0) mhz.push_back((double)(h[4 * b + 1] - h[4 * b + 0]) / dns * 1e3);
      }
      std::sort(mhz.begin(), mhz.end());
      *sm_mhz = mhz.empty() ? 0.0 : mhz[mhz.size() / 2];
    }
  }
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  cudaFree(sink);
  cudaFree(stamps);
  return rc;
}
