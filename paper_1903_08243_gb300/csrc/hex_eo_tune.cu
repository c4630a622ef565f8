// Even-odd FP64 instantiations with non-default cells per block (128- and
// 512-thread targets; hex_eo_cb_options lists them).  This unit has its own
// copy of the split tables in its constant bank.
#include "hex_eo.cuh"

namespace mfa {
namespace {

using namespace hexeo;

template <int N, int CBX>
cudaError_t dispatch_cb(int kind, bool colour, const HexApplyArgs& a, GridBudget budget, cudaStream_t s) {
  switch (kind) {
    case MFA_FORM_MASS:
      return colour ? launch<N, MFA_FORM_MASS, true, CBX>(a, budget, s)
                    : launch<N, MFA_FORM_MASS, false, CBX>(a, budget, s);
    case MFA_FORM_LAPLACE:
      return colour ? launch<N, MFA_FORM_LAPLACE, true, CBX>(a, budget, s)
                    : launch<N, MFA_FORM_LAPLACE, false, CBX>(a, budget, s);
    case MFA_FORM_HELMHOLTZ:
      return colour ? launch<N, MFA_FORM_HELMHOLTZ, true, CBX>(a, budget, s)
                    : launch<N, MFA_FORM_HELMHOLTZ, false, CBX>(a, budget, s);
  }
  return cudaErrorInvalidValue;
}

template <int N>
cudaError_t dispatch_target(int kind, bool colour, int cb, const HexApplyArgs& a, GridBudget budget, cudaStream_t s) {
  constexpr int lo = eo_cb_for(N, 128), hi = eo_cb_for(N, 512);
  static_assert(lo != eo_cb_for(N, 256) && hi != eo_cb_for(N, 256), "tuned choices differ from the default");
  if (cb == lo) return dispatch_cb<N, lo>(kind, colour, a, budget, s);
  if (cb == hi) return dispatch_cb<N, hi>(kind, colour, a, budget, s);
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t hex_eo_apply_launch_cb(int n, int kind, bool colour, int cb, const HexApplyArgs& a, GridBudget budget,
                                   cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  switch (n) {
    case 5: return dispatch_target<5>(kind, colour, cb, a, budget, s);
    case 6: return dispatch_target<6>(kind, colour, cb, a, budget, s);
    case 7: return dispatch_target<7>(kind, colour, cb, a, budget, s);
    case 8: return dispatch_target<8>(kind, colour, cb, a, budget, s);
    case 9: return dispatch_target<9>(kind, colour, cb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mfa
