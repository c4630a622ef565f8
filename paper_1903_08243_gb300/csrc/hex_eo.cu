// Instantiations and launchers of the even-odd FP64 hex action (hex_eo.cuh).
#include <mutex>
#include <vector>

#include "hex_eo.cuh"

namespace mfa {
namespace {

using namespace hexeo;

std::mutex g_mutex;
bool g_ready[64] = {false};

// Split tables of B, B^T, D, D^T for n = 5..9 into this unit's constant bank.
cudaError_t upload_tables() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_ready[dev]) return cudaSuccess;
  std::vector<double> tab(kTabDoubles, 0.0);
  for (int n = 5; n <= 9; ++n) {
    double gll[kMaxN], xg[kMaxN], wg[kMaxN], B[kMaxN * kMaxN], D[kMaxN * kMaxN];
    gll01(n, gll);
    gauss_legendre01(n, xg, wg);
    lagrange_matrix(n, gll, n, xg, B);  // B[q][a]
    collocation_derivative(n, xg, D);   // D[q][r]
    const int h = n / 2;
    for (int mat = 0; mat < 4; ++mat) {
      auto S = [&](int i, int j) {
        const double* M = mat < 2 ? B : D;
        return (mat % 2 == 0) ? M[i * n + j] : M[j * n + i];  // odd mat: transpose
      };
      double* o = tab.data() + tab_offset(n, mat);
      for (int i = 0; i < h; ++i)
        for (int j = 0; j < h; ++j) {
          o[i * h + j] = 0.5 * (S(i, j) + S(i, n - 1 - j));              // E
          o[h * h + i * h + j] = 0.5 * (S(i, j) - S(i, n - 1 - j));      // O
        }
      if (n & 1) {
        for (int i = 0; i < h; ++i) o[2 * h * h + i] = S(i, h);          // Mc
        for (int j = 0; j <= h; ++j) o[2 * h * h + h + j] = S(h, j);     // Mr
      }
    }
  }
  e = cudaMemcpyToSymbol(c_eo, tab.data(), sizeof(double) * kTabDoubles);
  if (e == cudaSuccess) g_ready[dev] = true;
  return e;
}

template <typename Kern>
int occupancy(Kern kern, int threads, int smem) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int b = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem) != cudaSuccess || b < 1) b = 1;
  return b;
}

template <int N, int KIND, bool COLOUR>
cudaError_t launch(const HexApplyArgs& a, int sm_count, cudaStream_t s) {
  using S = EShape<N>;
  auto kern = eo_apply_kernel<N, KIND, COLOUR>;
  static int bps = -1;
  if (bps < 0) bps = occupancy(kern, S::T, S::SMEM);
  const int64_t nbatch = (a.count + S::CB - 1) / S::CB;
  if (nbatch == 0) return cudaSuccess;
  const int64_t cap = (int64_t)sm_count * bps;
  kern<<<(unsigned)(nbatch < cap ? nbatch : cap), S::T, S::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <int N, int KIND>
cudaError_t launch_group(const HexApplyArgs* items, const int64_t* first, int nitems, int64_t total, int sm_count,
                         cudaStream_t s) {
  using S = EShape<N>;
  auto kern = eo_group_kernel<N, KIND>;
  static int bps = -1;
  if (bps < 0) bps = occupancy(kern, S::T, S::SMEM);
  if (total == 0) return cudaSuccess;
  const int64_t cap = (int64_t)sm_count * bps;
  kern<<<(unsigned)(total < cap ? total : cap), S::T, S::SMEM, s>>>(items, first, nitems);
  return cudaGetLastError();
}

template <int N>
cudaError_t dispatch(int kind, bool colour, const HexApplyArgs& a, int sm_count, cudaStream_t s) {
  switch (kind) {
    case MFA_FORM_MASS:
      return colour ? launch<N, MFA_FORM_MASS, true>(a, sm_count, s) : launch<N, MFA_FORM_MASS, false>(a, sm_count, s);
    case MFA_FORM_LAPLACE:
      return colour ? launch<N, MFA_FORM_LAPLACE, true>(a, sm_count, s)
                    : launch<N, MFA_FORM_LAPLACE, false>(a, sm_count, s);
    case MFA_FORM_HELMHOLTZ:
      return colour ? launch<N, MFA_FORM_HELMHOLTZ, true>(a, sm_count, s)
                    : launch<N, MFA_FORM_HELMHOLTZ, false>(a, sm_count, s);
  }
  return cudaErrorInvalidValue;
}

template <int N>
cudaError_t dispatch_group(int kind, const HexApplyArgs* items, const int64_t* first, int nitems, int64_t total,
                           int sm_count, cudaStream_t s) {
  switch (kind) {
    case MFA_FORM_MASS: return launch_group<N, MFA_FORM_MASS>(items, first, nitems, total, sm_count, s);
    case MFA_FORM_LAPLACE: return launch_group<N, MFA_FORM_LAPLACE>(items, first, nitems, total, sm_count, s);
    case MFA_FORM_HELMHOLTZ: return launch_group<N, MFA_FORM_HELMHOLTZ>(items, first, nitems, total, sm_count, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int hex_eo_cells_per_block(int n) {
  const int l = n * n;
  return 256 / l > 0 ? 256 / l : 1;  // hexeo::EShape<N>::CB
}

cudaError_t hex_eo_apply_launch(int n, int kind, bool colour, const HexApplyArgs& a, int sm_count, cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  switch (n) {
    case 5: return dispatch<5>(kind, colour, a, sm_count, s);
    case 6: return dispatch<6>(kind, colour, a, sm_count, s);
    case 7: return dispatch<7>(kind, colour, a, sm_count, s);
    case 8: return dispatch<8>(kind, colour, a, sm_count, s);
    case 9: return dispatch<9>(kind, colour, a, sm_count, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t hex_eo_group_launch(int n, int kind, const HexApplyArgs* items, const int64_t* first, int nitems,
                                int64_t total, int sm_count, cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  switch (n) {
    case 5: return dispatch_group<5>(kind, items, first, nitems, total, sm_count, s);
    case 6: return dispatch_group<6>(kind, items, first, nitems, total, sm_count, s);
    case 7: return dispatch_group<7>(kind, items, first, nitems, total, sm_count, s);
    case 8: return dispatch_group<8>(kind, items, first, nitems, total, sm_count, s);
    case 9: return dispatch_group<9>(kind, items, first, nitems, total, sm_count, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mfa
