// Instantiations of the sum-factorised hex action for the FP32 and BF16
// variants (compiled separately from the FP64 ones to build in parallel).
#include "hex_kernels.cuh"

namespace mfa {

cudaError_t hex_apply_launch_mixed(int n, int nq, int kind, int prec, bool colour, const HexTables& tb,
                                   const HexApplyArgs& a, int sm_count, cudaStream_t s) {
  using namespace hexk;
  if (prec == MFA_PREC_FP32) {
    MFA_HEX_KIND_CASES(2, 2, MFA_PREC_FP32)
    MFA_HEX_KIND_CASES(3, 3, MFA_PREC_FP32)
    MFA_HEX_KIND_CASES(4, 4, MFA_PREC_FP32)
    MFA_HEX_KIND_CASES(5, 5, MFA_PREC_FP32)
    MFA_HEX_KIND_CASES(6, 6, MFA_PREC_FP32)
    MFA_HEX_KIND_CASES(7, 7, MFA_PREC_FP32)
    MFA_HEX_KIND_CASES(8, 8, MFA_PREC_FP32)
    MFA_HEX_KIND_CASES(9, 9, MFA_PREC_FP32)
  } else if (prec == MFA_PREC_BF16) {
    MFA_HEX_KIND_CASES(2, 2, MFA_PREC_BF16)
    MFA_HEX_KIND_CASES(3, 3, MFA_PREC_BF16)
    MFA_HEX_KIND_CASES(4, 4, MFA_PREC_BF16)
    MFA_HEX_KIND_CASES(5, 5, MFA_PREC_BF16)
    MFA_HEX_KIND_CASES(6, 6, MFA_PREC_BF16)
    MFA_HEX_KIND_CASES(7, 7, MFA_PREC_BF16)
    MFA_HEX_KIND_CASES(8, 8, MFA_PREC_BF16)
    MFA_HEX_KIND_CASES(9, 9, MFA_PREC_BF16)
  }
  return cudaErrorInvalidValue;
}

cudaError_t hex_group_launch_mixed(int n, int kind, int prec, const HexTables& tb, const HexApplyArgs* items,
                                   const int64_t* first, int nitems, int64_t total, int sm_count, cudaStream_t s) {
  using namespace hexk;
  if (prec == MFA_PREC_FP32) {
    MFA_HEX_GROUP_CASES(2, MFA_PREC_FP32)
    MFA_HEX_GROUP_CASES(3, MFA_PREC_FP32)
    MFA_HEX_GROUP_CASES(4, MFA_PREC_FP32)
    MFA_HEX_GROUP_CASES(5, MFA_PREC_FP32)
    MFA_HEX_GROUP_CASES(6, MFA_PREC_FP32)
    MFA_HEX_GROUP_CASES(7, MFA_PREC_FP32)
    MFA_HEX_GROUP_CASES(8, MFA_PREC_FP32)
    MFA_HEX_GROUP_CASES(9, MFA_PREC_FP32)
  } else if (prec == MFA_PREC_BF16) {
    MFA_HEX_GROUP_CASES(2, MFA_PREC_BF16)
    MFA_HEX_GROUP_CASES(3, MFA_PREC_BF16)
    MFA_HEX_GROUP_CASES(4, MFA_PREC_BF16)
    MFA_HEX_GROUP_CASES(5, MFA_PREC_BF16)
    MFA_HEX_GROUP_CASES(6, MFA_PREC_BF16)
    MFA_HEX_GROUP_CASES(7, MFA_PREC_BF16)
    MFA_HEX_GROUP_CASES(8, MFA_PREC_BF16)
    MFA_HEX_GROUP_CASES(9, MFA_PREC_BF16)
  }
  return cudaErrorInvalidValue;
}

}  // namespace mfa
