// FP32/BF16 line-kernel instantiations for n = 2..5 with the
// non-default staging choice and/or the 512-thread block target (the
// autotuner's choices; double vectors only).  This unit has its own copy of
// the 1D tables in its constant bank.
#include "hex_lines.cuh"

namespace mfa {
using namespace hexl;
namespace {

template <int N, int KIND, int PREC>
cudaError_t tuned(bool stg, int cb, const LineArgs& a, GridBudget budget, cudaStream_t s) {
  constexpr bool D = staged<PREC>();
  constexpr int C0 = line_cb_for(N, 256), C1 = line_cb_for(N, 512);
  static_assert(C0 != C1, "the 512-thread target differs from the default");
  if (stg != D && cb == C0) return launch_line<N, KIND, PREC, double, !D, C0>(a, budget, s);
  if (stg == D && cb == C1) return launch_line<N, KIND, PREC, double, D, C1>(a, budget, s);
  if (stg != D && cb == C1) return launch_line<N, KIND, PREC, double, !D, C1>(a, budget, s);
  return cudaErrorInvalidValue;  // the default lives in hex_lines_a.cu
}

template <int N>
cudaError_t tuned_kind(int kind, int prec, bool stg, int cb, const LineArgs& a, GridBudget budget, cudaStream_t s) {
  const bool bf = prec == MFA_PREC_BF16;
  switch (kind) {
    case MFA_FORM_MASS:
      return bf ? tuned<N, MFA_FORM_MASS, MFA_PREC_BF16>(stg, cb, a, budget, s)
                : tuned<N, MFA_FORM_MASS, MFA_PREC_FP32>(stg, cb, a, budget, s);
    case MFA_FORM_LAPLACE:
      return bf ? tuned<N, MFA_FORM_LAPLACE, MFA_PREC_BF16>(stg, cb, a, budget, s)
                : tuned<N, MFA_FORM_LAPLACE, MFA_PREC_FP32>(stg, cb, a, budget, s);
    case MFA_FORM_HELMHOLTZ:
      return bf ? tuned<N, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16>(stg, cb, a, budget, s)
                : tuned<N, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32>(stg, cb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t hex_line_tuned_a(int n, int kind, int prec, bool stg, int cb, const LineArgs& a, GridBudget budget,
                             cudaStream_t s) {
  if (prec != MFA_PREC_FP32 && prec != MFA_PREC_BF16) return cudaErrorInvalidValue;
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  switch (n) {
    case 2: return tuned_kind<2>(kind, prec, stg, cb, a, budget, s);
    case 3: return tuned_kind<3>(kind, prec, stg, cb, a, budget, s);
    case 4: return tuned_kind<4>(kind, prec, stg, cb, a, budget, s);
    case 5: return tuned_kind<5>(kind, prec, stg, cb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mfa
