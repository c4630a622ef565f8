// FP64 point-kernel instantiations with non-default cells per block (the
// autotuner's choices for p+1 points; hex_point_cb_options lists them).
#include "hex_kernels.cuh"

namespace mfa {

cudaError_t hex_point_launch_cb(int n, int nq, int kind, bool colour, int cb, const HexTables& tb,
                                const HexApplyArgs& a, GridBudget budget, cudaStream_t s) {
  using namespace hexk;
  MFA_HEX_KIND_CASES_CB(2, 2, 16, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES_CB(2, 2, 64, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES_CB(3, 3, 4, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES_CB(3, 3, 18, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES_CB(4, 4, 2, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES_CB(4, 4, 8, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES_CB(5, 5, 1, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES_CB(5, 5, 4, MFA_PREC_FP64)
  MFA_HEX_KIND_CASES_CB(6, 6, 2, MFA_PREC_FP64)
  return cudaErrorInvalidValue;
}

}  // namespace mfa
