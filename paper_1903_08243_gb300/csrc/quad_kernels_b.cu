// Instantiations of the quadrilateral action for n = 6..9 (quad_kernels.cuh).
#include "quad_kernels.cuh"

namespace mfa {

cudaError_t quad_apply_launch_b(int n, int nq, int ncomp, int kind, int law, bool colour, const HexTables& tb,
                                const QuadArgs& a, GridBudget budget, cudaStream_t s) {
  switch (n) {
    case 6: return by_rule<6>(nq, ncomp, kind, law, colour, tb, a, budget, s);
    case 7: return by_rule<7>(nq, ncomp, kind, law, colour, tb, a, budget, s);
    case 8: return by_rule<8>(nq, ncomp, kind, law, colour, tb, a, budget, s);
    case 9: return by_rule<9>(nq, ncomp, kind, law, colour, tb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mfa
