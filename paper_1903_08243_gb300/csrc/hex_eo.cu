// Instantiations and launchers of the even-odd FP64 hex action (hex_eo.cuh).
#include "hex_eo.cuh"

namespace mfa {
namespace {

using namespace hexeo;

template <int N, int KIND>
cudaError_t launch_group(const HexApplyArgs* items, const int64_t* first, int nitems, int64_t total, GridBudget budget,
                         cudaStream_t s) {
  using S = EShape<N>;
  auto kern = eo_group_kernel<N, KIND>;
  static int bps = -1;
  if (bps < 0) bps = occupancy(kern, S::T, S::SMEM);
  if (total == 0) return cudaSuccess;
  const int64_t cap = budget.cap(bps);
  kern<<<(unsigned)(total < cap ? total : cap), S::T, S::SMEM, s>>>(items, first, nitems);
  return cudaGetLastError();
}

template <int N>
cudaError_t dispatch(int kind, bool colour, const HexApplyArgs& a, GridBudget budget, cudaStream_t s) {
  switch (kind) {
    case MFA_FORM_MASS:
      return colour ? launch<N, MFA_FORM_MASS, true>(a, budget, s) : launch<N, MFA_FORM_MASS, false>(a, budget, s);
    case MFA_FORM_LAPLACE:
      return colour ? launch<N, MFA_FORM_LAPLACE, true>(a, budget, s)
                    : launch<N, MFA_FORM_LAPLACE, false>(a, budget, s);
    case MFA_FORM_HELMHOLTZ:
      return colour ? launch<N, MFA_FORM_HELMHOLTZ, true>(a, budget, s)
                    : launch<N, MFA_FORM_HELMHOLTZ, false>(a, budget, s);
  }
  return cudaErrorInvalidValue;
}

template <int N>
cudaError_t dispatch_group(int kind, const HexApplyArgs* items, const int64_t* first, int nitems, int64_t total,
                           GridBudget budget, cudaStream_t s) {
  switch (kind) {
    case MFA_FORM_MASS: return launch_group<N, MFA_FORM_MASS>(items, first, nitems, total, budget, s);
    case MFA_FORM_LAPLACE: return launch_group<N, MFA_FORM_LAPLACE>(items, first, nitems, total, budget, s);
    case MFA_FORM_HELMHOLTZ: return launch_group<N, MFA_FORM_HELMHOLTZ>(items, first, nitems, total, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int hex_eo_cells_per_block(int n) { return eo_cb_for(n, 256); }  // hexeo::EShape<N>::CB

// Default (256-thread target), then 128- and 512-thread targets (hex_eo_tune.cu).
int hex_eo_cb_options(int n, int* out) {
  if (n < 5 || n > 9) return 0;
  out[0] = eo_cb_for(n, 256);
  out[1] = eo_cb_for(n, 128);
  out[2] = eo_cb_for(n, 512);
  return 3;
}

cudaError_t hex_eo_apply_launch(int n, int kind, bool colour, const HexApplyArgs& a, GridBudget budget, cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  switch (n) {
    case 5: return dispatch<5>(kind, colour, a, budget, s);
    case 6: return dispatch<6>(kind, colour, a, budget, s);
    case 7: return dispatch<7>(kind, colour, a, budget, s);
    case 8: return dispatch<8>(kind, colour, a, budget, s);
    case 9: return dispatch<9>(kind, colour, a, budget, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t hex_eo_group_launch(int n, int kind, const HexApplyArgs* items, const int64_t* first, int nitems,
                                int64_t total, GridBudget budget, cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  switch (n) {
    case 5: return dispatch_group<5>(kind, items, first, nitems, total, budget, s);
    case 6: return dispatch_group<6>(kind, items, first, nitems, total, budget, s);
    case 7: return dispatch_group<7>(kind, items, first, nitems, total, budget, s);
    case 8: return dispatch_group<8>(kind, items, first, nitems, total, budget, s);
    case 9: return dispatch_group<9>(kind, items, first, nitems, total, budget, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mfa
