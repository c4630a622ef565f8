// Halo buffers of a cell-partitioned operator action.
//
// Section 2.2's global assembly adds every cell's local result into the dofs
// that the cell touches.  With the cells split over ranks, a node touched by
// cells of several ranks is owned by one of them and held as a ghost by the
// others.  One distributed apply imports x at the ghosts from the owners,
// applies the rank's cells, and adds the ghosts' partial sums into the
// owners' entries (the reverse exchange).  These kernels move values between
// a rank's node vectors and the contiguous buffers that the exchange sends
// and receives: pack gathers v at a list of nodes, unpack writes or adds a
// buffer back at a list of nodes.
#include <cstdio>

#include "mfa_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kErrRange = 8;  // error flag bit: an index outside [0, nnode)

__global__ void halo_pack_kernel(const int32_t* __restrict__ ids, int64_t n, int nc, int64_t nnode,
                                 const double* __restrict__ v, double* __restrict__ buf, int* err) {
  const int64_t total = n * nc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / nc;
    const int c = (int)(i - k * nc);
    const int32_t id = __ldg(ids + k);
    if (id < 0 || id >= nnode) {
      atomicOr(err, kErrRange);
      buf[i] = 0.0;
      continue;
    }
    buf[i] = __ldg(v + (int64_t)id * nc + c);
  }
}

template <bool ACC>
__global__ void halo_unpack_kernel(const int32_t* __restrict__ ids, int64_t n, int nc, int64_t nnode,
                                   const double* __restrict__ buf, double* __restrict__ v, int* err) {
  const int64_t total = n * nc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i / nc;
    const int c = (int)(i - k * nc);
    const int32_t id = __ldg(ids + k);
    if (id < 0 || id >= nnode) {
      atomicOr(err, kErrRange);
      continue;
    }
    double* dst = v + (int64_t)id * nc + c;
    if (ACC) *dst += buf[i];
    else *dst = buf[i];
  }
}

int check(mfa_ctx* ctx, const int32_t* ids, int64_t n, int ncomp, int64_t nnode, const void* a, const void* b,
          const char* name) {
  if (!ctx || n < 0 || ncomp < 1 || nnode < 0 || (n > 0 && (!ids || !a || !b))) {
    char msg[96];
    snprintf(msg, sizeof(msg), "%s: bad argument", name);
    return mfa::set_error(MFA_ERR_ARG, msg);
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return mfa::set_error(MFA_ERR_CUDA, "halo: cudaSetDevice");
  mfa::clear_stale_error();
  return MFA_OK;
}

unsigned blocks_for(const mfa_ctx* ctx, int64_t total) {
  const int64_t want = (total + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)ctx->sm_count * 8;
  return (unsigned)(want < cap ? want : cap);
}

}  // namespace

extern "C" int mfa_halo_pack(mfa_ctx* ctx, const int32_t* ids, int64_t n, int ncomp, int64_t nnode, const double* v,
                             double* buf) {
  int rc = check(ctx, ids, n, ncomp, nnode, v, buf, "mfa_halo_pack");
  if (rc || n == 0) return rc;
  halo_pack_kernel<<<blocks_for(ctx, n * ncomp), kThreads, 0, ctx->stream>>>(ids, n, ncomp, nnode, v, buf,
                                                                            ctx->d_err);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MFA_OK : mfa::set_error(MFA_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" int mfa_halo_unpack(mfa_ctx* ctx, const int32_t* ids, int64_t n, int ncomp, int64_t nnode,
                               const double* buf, double* v, int accumulate) {
  int rc = check(ctx, ids, n, ncomp, nnode, buf, v, "mfa_halo_unpack");
  if (rc || n == 0) return rc;
  const unsigned grid = blocks_for(ctx, n * ncomp);
  if (accumulate)
    halo_unpack_kernel<true><<<grid, kThreads, 0, ctx->stream>>>(ids, n, ncomp, nnode, buf, v, ctx->d_err);
  else
    halo_unpack_kernel<false><<<grid, kThreads, 0, ctx->stream>>>(ids, n, ncomp, nnode, buf, v, ctx->d_err);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MFA_OK : mfa::set_error(MFA_ERR_CUDA, cudaGetErrorString(e));
}
