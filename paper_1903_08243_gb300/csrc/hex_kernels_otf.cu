// FP64 point-kernel instantiations with the geometry recomputed at every Gauss point from the cell's
// vertices (the paper's choice for trilinear cells, Section 4.1), p+1 points, default cells per block.
#include "hex_kernels.cuh"

namespace mfa {
namespace {

template <int N>
cudaError_t otf_kind(int kind, bool colour, const HexTables& tb, const HexApplyArgs& a, GridBudget budget, cudaStream_t s) {
  using namespace hexk;
  switch (kind) {
    case MFA_FORM_MASS:
      return colour ? launch_apply<N, N, MFA_FORM_MASS, true, MFA_PREC_FP64, 0, false, true>(tb, a, budget, s)
                    : launch_apply<N, N, MFA_FORM_MASS, false, MFA_PREC_FP64, 0, false, true>(tb, a, budget, s);
    case MFA_FORM_LAPLACE:
      return colour ? launch_apply<N, N, MFA_FORM_LAPLACE, true, MFA_PREC_FP64, 0, false, true>(tb, a, budget, s)
                    : launch_apply<N, N, MFA_FORM_LAPLACE, false, MFA_PREC_FP64, 0, false, true>(tb, a, budget, s);
    case MFA_FORM_HELMHOLTZ:
      return colour ? launch_apply<N, N, MFA_FORM_HELMHOLTZ, true, MFA_PREC_FP64, 0, false, true>(tb, a, budget, s)
                    : launch_apply<N, N, MFA_FORM_HELMHOLTZ, false, MFA_PREC_FP64, 0, false, true>(tb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t hex_point_launch_otf(int n, int nq, int kind, bool colour, const HexTables& tb, const HexApplyArgs& a,
                                 GridBudget budget, cudaStream_t s) {
  if (nq != n || !a.coords || !a.cell_vert) return cudaErrorInvalidValue;
  switch (n) {
    case 2: return otf_kind<2>(kind, colour, tb, a, budget, s);
    case 3: return otf_kind<3>(kind, colour, tb, a, budget, s);
    case 4: return otf_kind<4>(kind, colour, tb, a, budget, s);
    case 5: return otf_kind<5>(kind, colour, tb, a, budget, s);
    case 6: return otf_kind<6>(kind, colour, tb, a, budget, s);
    case 7: return otf_kind<7>(kind, colour, tb, a, budget, s);
    case 8: return otf_kind<8>(kind, colour, tb, a, budget, s);
    case 9: return otf_kind<9>(kind, colour, tb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mfa
