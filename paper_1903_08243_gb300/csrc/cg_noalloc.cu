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
// so the address is queried once per device and cached.
int scratch_for(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return MFA_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[device]) {
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
  int rc = scratch_for(ctx->device, &base);
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

  auto dot = [&](const double* u, const double* v, double* out) -> int {
    cudaError_t e = mfa::dot_launch(u, v, n, partial, dres, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dres, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
  };
  auto precondition = [&](const double* in, double* outv) -> int {
    cudaError_t e = precond == MFA_PC_JACOBI ? mfa::pointwise_mul_launch(dinv, in, outv, n, s)
                                             : cudaMemcpyAsync(outv, in, n * 8, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
  };

  int it = 0;
  double bnorm = 0.0, rr = 0.0, rz = 0.0, res = 0.0;
  if (precond == MFA_PC_JACOBI) {
    rc = mfa_diagonal(ctx, f, dinv);
    if (!rc && mfa::reciprocal_launch(dinv, dinv, n, s) != cudaSuccess) rc = MFA_ERR_CUDA;
  }
  if (!rc) rc = dot(b, b, &bnorm);
  if (!rc) {
    bnorm = std::sqrt(bnorm);
    rc = mfa_apply(ctx, f, x, r, 0);
  }
  if (!rc && mfa::axpby_launch(1.0, b, -1.0, r, n, s) != cudaSuccess) rc = MFA_ERR_CUDA;
  if (!rc) rc = dot(r, r, &rr);
  if (!rc) rc = precondition(r, z);
  if (!rc) rc = dot(r, z, &rz);
  if (!rc && cudaMemcpyAsync(p, z, n * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess) rc = MFA_ERR_CUDA;
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
    if (mfa::axpby_launch(alpha, p, 1.0, x, n, s) != cudaSuccess ||
        mfa::axpby_launch(-alpha, q, 1.0, r, n, s) != cudaSuccess) {
      rc = MFA_ERR_CUDA;
      break;
    }
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
    if (mfa::axpby_launch(1.0, z, beta, p, n, s) != cudaSuccess) {
      rc = MFA_ERR_CUDA;
      break;
    }
  }
  if (!rc) rc = mfa_sync(ctx);
  if (rc == MFA_ERR_BREAKDOWN) mfa::set_error(rc, "mfa_cg_noalloc: breakdown (p.Ap <= 0 or a non-finite scalar)");
  if (rc == MFA_ERR_CUDA) mfa::set_error(rc, "mfa_cg_noalloc: a CUDA call failed");
  if (!rc && res > rtol) rc = mfa::set_error(MFA_ERR_NOT_CONVERGED, "mfa_cg_noalloc: not converged");
  if (iters) *iters = it;
  if (relres) *relres = res;
  return rc;
}
