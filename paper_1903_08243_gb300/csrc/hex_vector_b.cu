// Instantiations of the FP64 hex vector-form action for n = 6..9 (hex_vector.cuh).
#include "hex_vector.cuh"

namespace mfa {

cudaError_t hex_vector_launch_b(int n, int nq, int kind, int law, bool colour, const HexTables& tb, const HexVecArgs& a,
                                GridBudget budget, cudaStream_t s) {
  switch (n) {
    case 6: return hexv::dispatch<6>(nq, kind, law, colour, tb, a, budget, s);
    case 7: return hexv::dispatch<7>(nq, kind, law, colour, tb, a, budget, s);
    case 8: return hexv::dispatch<8>(nq, kind, law, colour, tb, a, budget, s);
    case 9: return hexv::dispatch<9>(nq, kind, law, colour, tb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mfa
