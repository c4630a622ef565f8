// Instantiations of the quadrilateral action for n = 2..5 (quad_kernels.cuh).
#include "quad_kernels.cuh"

namespace mfa {

cudaError_t quad_apply_launch_a(int n, int nq, int ncomp, int kind, int law, bool colour, const HexTables& tb,
                                const QuadArgs& a, GridBudget budget, cudaStream_t s) {
  switch (n) {
    case 2: return by_rule<2>(nq, ncomp, kind, law, colour, tb, a, budget, s);
    case 3: return by_rule<3>(nq, ncomp, kind, law, colour, tb, a, budget, s);
    case 4: return by_rule<4>(nq, ncomp, kind, law, colour, tb, a, budget, s);
    case 5: return by_rule<5>(nq, ncomp, kind, law, colour, tb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mfa
