// FP64 point-kernel instantiations with the warp-aggregated atomic scatter
// (p+1 points, default cells per block).
#include "hex_kernels.cuh"

namespace mfa {
namespace {

template <int N>
cudaError_t agg_kind(int kind, const HexTables& tb, const HexApplyArgs& a, GridBudget budget, cudaStream_t s) {
  using namespace hexk;
  switch (kind) {
    case MFA_FORM_MASS: return launch_apply<N, N, MFA_FORM_MASS, false, MFA_PREC_FP64, 0, true>(tb, a, budget, s);
    case MFA_FORM_LAPLACE:
      return launch_apply<N, N, MFA_FORM_LAPLACE, false, MFA_PREC_FP64, 0, true>(tb, a, budget, s);
    case MFA_FORM_HELMHOLTZ:
      return launch_apply<N, N, MFA_FORM_HELMHOLTZ, false, MFA_PREC_FP64, 0, true>(tb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t hex_point_launch_agg(int n, int nq, int kind, const HexTables& tb, const HexApplyArgs& a, GridBudget budget,
                                 cudaStream_t s) {
  if (nq != n) return cudaErrorInvalidValue;
  switch (n) {
    case 2: return agg_kind<2>(kind, tb, a, budget, s);
    case 3: return agg_kind<3>(kind, tb, a, budget, s);
    case 4: return agg_kind<4>(kind, tb, a, budget, s);
    case 5: return agg_kind<5>(kind, tb, a, budget, s);
    case 6: return agg_kind<6>(kind, tb, a, budget, s);
    case 7: return agg_kind<7>(kind, tb, a, budget, s);
    case 8: return agg_kind<8>(kind, tb, a, budget, s);
    case 9: return agg_kind<9>(kind, tb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mfa
