// mfa_cg_noalloc: Jacobi-PCG / CG that allocates no device memory.
//
// Some callers cannot call cudaMalloc: an application whose memory pool
// already owns the device memory it may use, a solver step embedded in
// another framework's stream pipeline where the implicit device-wide
// synchronisation of cudaMalloc/cudaFree would stall unrelated work, or a
// control loop that forbids allocation after start-up.  mfa_cg allocates its
// five work vectors on every call; this variant takes them from one
// file-scope __device__ array instead.  The algorithm and every kernel are
// those of mfa_cg.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "mfa_internal.h"

namespace {

constexpr int64_t kMaxNdof = MFA_CG_NOALLOC_MAX_NDOF;
constexpr int kPartials = 1024;  // equals mfa::dot_partials(), checked at set-up
constexpr int64_t kScratchDoubles = 5 * kMaxNdof + kPartials + 32;

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) double g_cg_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (which must be current).
// In host code `g_cg_scratch` names a host-side stand-in, not device memory,
// so the address comes from cudaGetSymbolAddress.  The first call on a device
// looks it up and caches it.  Later calls look it up again whenever `s` is
// not capturing (a reset of the device gives the array a new address) and use
// the cached one while `s` captures.
int scratch_for(int device, cudaStream_t s, double** out) {
  if (device < 0 || device >= kMaxDevices) return MFA_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mutex);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone;
  if (capturing) (void)cudaGetLastError();  // a refused query is not sticky; treat it as a capture
  if (!capturing || !g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_cg_scratch);
    if (e != cudaSuccess || !p) return MFA_ERR_CUDA;
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return MFA_OK;
}

}  // namespace

extern "C" int mfa_cg_noalloc(mfa_ctx* ctx, mfa_form* f, int precond, const double* b, double* x, double rtol,
                              int maxit, int* iters, double* relres) {
  if (!ctx || !f || !b || !x) return mfa::set_error(MFA_ERR_ARG, "mfa_cg_noalloc: NULL argument");
  if (precond != MFA_PC_NONE && precond != MFA_PC_JACOBI)
    return mfa::set_error(MFA_ERR_ARG, "mfa_cg_noalloc: unknown preconditioner");
  if (f->p.kind > MFA_FORM_ELASTICITY && f->p.kind != MFA_FORM_HYPER_JAC)
    return mfa::set_error(MFA_ERR_ARG, "mfa_cg_noalloc: the residual form is not linear");
  if (!(rtol > 0.0) || maxit < 0) return mfa::set_error(MFA_ERR_ARG, "mfa_cg_noalloc: bad rtol or maxit");
  const int64_t n = f->space->nnode * f->space->ncomp;
  if (n > kMaxNdof) {
    char msg[160];
    snprintf(msg, sizeof(msg), "mfa_cg_noalloc: %lld dofs exceed the limit of %lld (MFA_CG_NOALLOC_MAX_NDOF)",
             (long long)n, (long long)kMaxNdof);
    return mfa::set_error(MFA_ERR_ARG, msg);
  }
  if (mfa::dot_partials() != kPartials) return mfa::set_error(MFA_ERR_UNSUPPORTED, "mfa_cg_noalloc: dot layout");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return mfa::set_error(MFA_ERR_CUDA, "mfa_cg_noalloc: cudaSetDevice");
  double* base = nullptr;
  int rc = scratch_for(ctx->device, ctx->stream, &base);
  if (rc) return mfa::set_error(rc, "mfa_cg_noalloc: cudaGetSymbolAddress of the scratch array failed");
  // Every region below is fully written before it is read in each call
  // (r and q by mfa_apply, z by the preconditioner, p by a copy, dinv by
  // mfa_diagonal, the partials by the dot kernels), so nothing carries over.
  double* r = base;
  double* z = r + kMaxNdof;
  double* p = z + kMaxNdof;
  double* q = p + kMaxNdof;
  double* dinv = q + kMaxNdof;
  double* partial = dinv + kMaxNdof;
  double* dres = partial + kPartials;
  cudaStream_t s = ctx->stream;

  // This file's own launches, copies and waits report their failure here; the
  // statuses of mfa_apply, mfa_diagonal and mfa_sync keep the callee's message.
  auto own = [](cudaError_t e, const char* what) -> int {
    if (e == cudaSuccess) return MFA_OK;
    char msg[200];
    snprintf(msg, sizeof(msg), "mfa_cg_noalloc: %s: %s", what, cudaGetErrorString(e));
    return mfa::set_error(MFA_ERR_CUDA, msg);
  };
  auto dot = [&](const double* u, const double* v, double* out) -> int {
    cudaError_t e = mfa::dot_launch(u, v, n, partial, dres, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dres, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return own(e, "dot product");
  };
  auto precondition = [&](const double* in, double* outv) -> int {
    cudaError_t e = precond == MFA_PC_JACOBI ? mfa::pointwise_mul_launch(dinv, in, outv, n, s)
                                             : cudaMemcpyAsync(outv, in, n * 8, cudaMemcpyDeviceToDevice, s);
    return own(e, "preconditioner");
  };

  int it = 0;
  double bnorm = 0.0, rr = 0.0, rz = 0.0, res = 0.0;
  if (precond == MFA_PC_JACOBI) {
    rc = mfa_diagonal(ctx, f, dinv);
    if (!rc) rc = own(mfa::reciprocal_launch(dinv, dinv, n, s), "reciprocal of the diagonal");
  }
  if (!rc) rc = dot(b, b, &bnorm);
  if (!rc) {
    bnorm = std::sqrt(bnorm);
    rc = mfa_apply(ctx, f, x, r, 0);
  }
  if (!rc) rc = own(mfa::axpby_launch(1.0, b, -1.0, r, n, s), "initial residual");
  if (!rc) rc = dot(r, r, &rr);
  if (!rc) rc = precondition(r, z);
  if (!rc) rc = dot(r, z, &rz);
  if (!rc) rc = own(cudaMemcpyAsync(p, z, n * 8, cudaMemcpyDeviceToDevice, s), "first search direction");
  res = bnorm > 0.0 ? std::sqrt(rr) / bnorm : std::sqrt(rr);
  if (!rc && (!std::isfinite(bnorm) || !std::isfinite(rr) || !std::isfinite(rz))) rc = MFA_ERR_BREAKDOWN;
  while (!rc && res > rtol && it < maxit) {
    double pq = 0.0;
    rc = mfa_apply(ctx, f, p, q, 0);
    if (!rc) rc = dot(p, q, &pq);
    if (rc) break;
    if (!(pq > 0.0) || !std::isfinite(pq) || !std::isfinite(rz)) {
      rc = MFA_ERR_BREAKDOWN;
      break;
    }
    const double alpha = rz / pq;
    rc = own(mfa::axpby_launch(alpha, p, 1.0, x, n, s), "solution update");
    if (!rc) rc = own(mfa::axpby_launch(-alpha, q, 1.0, r, n, s), "residual update");
    if (rc) break;
    rc = dot(r, r, &rr);
    ++it;
    if (rc) break;
    if (!std::isfinite(rr)) {
      rc = MFA_ERR_BREAKDOWN;
      break;
    }
    res = bnorm > 0.0 ? std::sqrt(rr) / bnorm : std::sqrt(rr);
    if (res <= rtol) break;
    double rz_new = 0.0;
    rc = precondition(r, z);
    if (!rc) rc = dot(r, z, &rz_new);
    if (rc) break;
    const double beta = rz_new / rz;
    rz = rz_new;
    rc = own(mfa::axpby_launch(1.0, z, beta, p, n, s), "search direction update");
    if (rc) break;
  }
  if (!rc) rc = mfa_sync(ctx);
  if (rc == MFA_ERR_BREAKDOWN) mfa::set_error(rc, "mfa_cg_noalloc: breakdown (p.Ap <= 0 or a non-finite scalar)");
  if (!rc && res > rtol) rc = mfa::set_error(MFA_ERR_NOT_CONVERGED, "mfa_cg_noalloc: not converged");
  if (iters) *iters = it;
  if (relres) *relres = res;
  return rc;
}
