// Instantiations of the FP64 hex vector-form action for n = 2..5 (hex_vector.cuh).
#include "hex_vector.cuh"

namespace mfa {

cudaError_t hex_vector_launch_a(int n, int nq, int kind, int law, bool colour, const HexTables& tb, const HexVecArgs& a,
                                GridBudget budget, cudaStream_t s) {
  switch (n) {
    case 2: return hexv::dispatch<2>(nq, kind, law, colour, tb, a, budget, s);
    case 3: return hexv::dispatch<3>(nq, kind, law, colour, tb, a, budget, s);
    case 4: return hexv::dispatch<4>(nq, kind, law, colour, tb, a, budget, s);
    case 5: return hexv::dispatch<5>(nq, kind, law, colour, tb, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mfa
