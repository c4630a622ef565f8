// Instantiations of the line-per-thread FP32/BF16 hex action for n = 2..5
// (the other degrees live in the sibling translation unit so both compile in parallel).
#include <mutex>
#include <vector>

#include "hex_lines.cuh"

namespace mfa {
namespace {

using namespace hexl;

std::mutex g_tab_mutex;
bool g_tab_ready[64] = {false};

// B (GLL basis at the Gauss points) and D (collocation derivative at the Gauss
// points) for every n, in float and rounded to bfloat16, into this unit's
// constant bank on the current device.
cudaError_t upload_tables() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_tab_mutex);
  if (g_tab_ready[dev]) return cudaSuccess;
  std::vector<float> tab(2 * kTabFloats, 0.0f);
  for (int n = 2; n <= 9; ++n) {
    double gll[kMaxN], xg[kMaxN], wg[kMaxN], B[kMaxN * kMaxN], D[kMaxN * kMaxN];
    gll01(n, gll);
    gauss_legendre01(n, xg, wg);
    lagrange_matrix(n, gll, n, xg, B);
    collocation_derivative(n, xg, D);
    const int off = tab_offset(n);
    for (int i = 0; i < n * n; ++i) {
      tab[off + i] = (float)B[i];
      tab[off + n * n + i] = (float)D[i];
      tab[kTabFloats + off + i] = __bfloat162float(__double2bfloat16(B[i]));
      tab[kTabFloats + off + n * n + i] = __bfloat162float(__double2bfloat16(D[i]));
    }
  }
  e = cudaMemcpyToSymbol(c_tab, tab.data(), sizeof(float) * 2 * kTabFloats);
  if (e == cudaSuccess) g_tab_ready[dev] = true;
  return e;
}

}  // namespace

cudaError_t hex_line_apply_a(int n, int kind, int prec, bool f32vec, const hexl::LineArgs& a, int sm_count,
                                 cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  if (n == 2 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<2, MFA_FORM_MASS, MFA_PREC_FP32, float>(a, sm_count, s)
                  : launch_line<2, MFA_FORM_MASS, MFA_PREC_FP32, double>(a, sm_count, s);
  if (n == 2 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<2, MFA_FORM_MASS, MFA_PREC_BF16, float>(a, sm_count, s)
                  : launch_line<2, MFA_FORM_MASS, MFA_PREC_BF16, double>(a, sm_count, s);
  if (n == 2 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<2, MFA_FORM_LAPLACE, MFA_PREC_FP32, float>(a, sm_count, s)
                  : launch_line<2, MFA_FORM_LAPLACE, MFA_PREC_FP32, double>(a, sm_count, s);
  if (n == 2 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<2, MFA_FORM_LAPLACE, MFA_PREC_BF16, float>(a, sm_count, s)
                  : launch_line<2, MFA_FORM_LAPLACE, MFA_PREC_BF16, double>(a, sm_count, s);
  if (n == 2 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<2, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, float>(a, sm_count, s)
                  : launch_line<2, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, double>(a, sm_count, s);
  if (n == 2 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<2, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, float>(a, sm_count, s)
                  : launch_line<2, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, double>(a, sm_count, s);
  if (n == 3 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<3, MFA_FORM_MASS, MFA_PREC_FP32, float>(a, sm_count, s)
                  : launch_line<3, MFA_FORM_MASS, MFA_PREC_FP32, double>(a, sm_count, s);
  if (n == 3 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<3, MFA_FORM_MASS, MFA_PREC_BF16, float>(a, sm_count, s)
                  : launch_line<3, MFA_FORM_MASS, MFA_PREC_BF16, double>(a, sm_count, s);
  if (n == 3 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<3, MFA_FORM_LAPLACE, MFA_PREC_FP32, float>(a, sm_count, s)
                  : launch_line<3, MFA_FORM_LAPLACE, MFA_PREC_FP32, double>(a, sm_count, s);
  if (n == 3 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<3, MFA_FORM_LAPLACE, MFA_PREC_BF16, float>(a, sm_count, s)
                  : launch_line<3, MFA_FORM_LAPLACE, MFA_PREC_BF16, double>(a, sm_count, s);
  if (n == 3 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<3, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, float>(a, sm_count, s)
                  : launch_line<3, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, double>(a, sm_count, s);
  if (n == 3 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<3, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, float>(a, sm_count, s)
                  : launch_line<3, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, double>(a, sm_count, s);
  if (n == 4 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<4, MFA_FORM_MASS, MFA_PREC_FP32, float>(a, sm_count, s)
                  : launch_line<4, MFA_FORM_MASS, MFA_PREC_FP32, double>(a, sm_count, s);
  if (n == 4 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<4, MFA_FORM_MASS, MFA_PREC_BF16, float>(a, sm_count, s)
                  : launch_line<4, MFA_FORM_MASS, MFA_PREC_BF16, double>(a, sm_count, s);
  if (n == 4 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<4, MFA_FORM_LAPLACE, MFA_PREC_FP32, float>(a, sm_count, s)
                  : launch_line<4, MFA_FORM_LAPLACE, MFA_PREC_FP32, double>(a, sm_count, s);
  if (n == 4 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<4, MFA_FORM_LAPLACE, MFA_PREC_BF16, float>(a, sm_count, s)
                  : launch_line<4, MFA_FORM_LAPLACE, MFA_PREC_BF16, double>(a, sm_count, s);
  if (n == 4 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<4, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, float>(a, sm_count, s)
                  : launch_line<4, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, double>(a, sm_count, s);
  if (n == 4 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<4, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, float>(a, sm_count, s)
                  : launch_line<4, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, double>(a, sm_count, s);
  if (n == 5 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<5, MFA_FORM_MASS, MFA_PREC_FP32, float>(a, sm_count, s)
                  : launch_line<5, MFA_FORM_MASS, MFA_PREC_FP32, double>(a, sm_count, s);
  if (n == 5 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<5, MFA_FORM_MASS, MFA_PREC_BF16, float>(a, sm_count, s)
                  : launch_line<5, MFA_FORM_MASS, MFA_PREC_BF16, double>(a, sm_count, s);
  if (n == 5 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<5, MFA_FORM_LAPLACE, MFA_PREC_FP32, float>(a, sm_count, s)
                  : launch_line<5, MFA_FORM_LAPLACE, MFA_PREC_FP32, double>(a, sm_count, s);
  if (n == 5 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<5, MFA_FORM_LAPLACE, MFA_PREC_BF16, float>(a, sm_count, s)
                  : launch_line<5, MFA_FORM_LAPLACE, MFA_PREC_BF16, double>(a, sm_count, s);
  if (n == 5 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<5, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, float>(a, sm_count, s)
                  : launch_line<5, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, double>(a, sm_count, s);
  if (n == 5 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<5, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, float>(a, sm_count, s)
                  : launch_line<5, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, double>(a, sm_count, s);
  return cudaErrorInvalidValue;
}

cudaError_t hex_line_group_a(int n, int kind, int prec, const HexApplyArgs* items, const int64_t* first,
                                 int nitems, int64_t total, int sm_count, cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  if (n == 2 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return launch_line_group<2, MFA_FORM_MASS, MFA_PREC_FP32>(items, first, nitems, total, sm_count, s);
  if (n == 2 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return launch_line_group<2, MFA_FORM_MASS, MFA_PREC_BF16>(items, first, nitems, total, sm_count, s);
  if (n == 2 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return launch_line_group<2, MFA_FORM_LAPLACE, MFA_PREC_FP32>(items, first, nitems, total, sm_count, s);
  if (n == 2 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return launch_line_group<2, MFA_FORM_LAPLACE, MFA_PREC_BF16>(items, first, nitems, total, sm_count, s);
  if (n == 2 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return launch_line_group<2, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32>(items, first, nitems, total, sm_count, s);
  if (n == 2 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return launch_line_group<2, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16>(items, first, nitems, total, sm_count, s);
  if (n == 3 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return launch_line_group<3, MFA_FORM_MASS, MFA_PREC_FP32>(items, first, nitems, total, sm_count, s);
  if (n == 3 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return launch_line_group<3, MFA_FORM_MASS, MFA_PREC_BF16>(items, first, nitems, total, sm_count, s);
  if (n == 3 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return launch_line_group<3, MFA_FORM_LAPLACE, MFA_PREC_FP32>(items, first, nitems, total, sm_count, s);
  if (n == 3 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return launch_line_group<3, MFA_FORM_LAPLACE, MFA_PREC_BF16>(items, first, nitems, total, sm_count, s);
  if (n == 3 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return launch_line_group<3, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32>(items, first, nitems, total, sm_count, s);
  if (n == 3 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return launch_line_group<3, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16>(items, first, nitems, total, sm_count, s);
  if (n == 4 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return launch_line_group<4, MFA_FORM_MASS, MFA_PREC_FP32>(items, first, nitems, total, sm_count, s);
  if (n == 4 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return launch_line_group<4, MFA_FORM_MASS, MFA_PREC_BF16>(items, first, nitems, total, sm_count, s);
  if (n == 4 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return launch_line_group<4, MFA_FORM_LAPLACE, MFA_PREC_FP32>(items, first, nitems, total, sm_count, s);
  if (n == 4 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return launch_line_group<4, MFA_FORM_LAPLACE, MFA_PREC_BF16>(items, first, nitems, total, sm_count, s);
  if (n == 4 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return launch_line_group<4, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32>(items, first, nitems, total, sm_count, s);
  if (n == 4 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return launch_line_group<4, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16>(items, first, nitems, total, sm_count, s);
  if (n == 5 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return launch_line_group<5, MFA_FORM_MASS, MFA_PREC_FP32>(items, first, nitems, total, sm_count, s);
  if (n == 5 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return launch_line_group<5, MFA_FORM_MASS, MFA_PREC_BF16>(items, first, nitems, total, sm_count, s);
  if (n == 5 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return launch_line_group<5, MFA_FORM_LAPLACE, MFA_PREC_FP32>(items, first, nitems, total, sm_count, s);
  if (n == 5 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return launch_line_group<5, MFA_FORM_LAPLACE, MFA_PREC_BF16>(items, first, nitems, total, sm_count, s);
  if (n == 5 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return launch_line_group<5, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32>(items, first, nitems, total, sm_count, s);
  if (n == 5 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return launch_line_group<5, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16>(items, first, nitems, total, sm_count, s);
  return cudaErrorInvalidValue;
}

}  // namespace mfa
