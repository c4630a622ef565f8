// Instantiations of the line-per-thread FP32/BF16 hex action for n = 2..5
// (the other degrees live in the sibling translation unit so both compile in parallel).
#include "hex_lines.cuh"

namespace mfa {
using namespace hexl;

cudaError_t hex_line_apply_a(int n, int kind, int prec, bool f32vec, const hexl::LineArgs& a, GridBudget budget,
                                 cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  if (n == 2 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<2, MFA_FORM_MASS, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<2, MFA_FORM_MASS, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 2 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<2, MFA_FORM_MASS, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<2, MFA_FORM_MASS, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 2 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<2, MFA_FORM_LAPLACE, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<2, MFA_FORM_LAPLACE, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 2 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<2, MFA_FORM_LAPLACE, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<2, MFA_FORM_LAPLACE, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 2 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<2, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<2, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 2 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<2, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<2, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 3 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<3, MFA_FORM_MASS, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<3, MFA_FORM_MASS, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 3 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<3, MFA_FORM_MASS, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<3, MFA_FORM_MASS, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 3 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<3, MFA_FORM_LAPLACE, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<3, MFA_FORM_LAPLACE, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 3 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<3, MFA_FORM_LAPLACE, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<3, MFA_FORM_LAPLACE, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 3 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<3, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<3, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 3 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<3, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<3, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 4 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<4, MFA_FORM_MASS, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<4, MFA_FORM_MASS, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 4 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<4, MFA_FORM_MASS, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<4, MFA_FORM_MASS, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 4 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<4, MFA_FORM_LAPLACE, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<4, MFA_FORM_LAPLACE, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 4 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<4, MFA_FORM_LAPLACE, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<4, MFA_FORM_LAPLACE, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 4 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<4, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<4, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 4 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<4, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<4, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 5 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<5, MFA_FORM_MASS, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<5, MFA_FORM_MASS, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 5 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<5, MFA_FORM_MASS, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<5, MFA_FORM_MASS, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 5 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<5, MFA_FORM_LAPLACE, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<5, MFA_FORM_LAPLACE, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 5 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<5, MFA_FORM_LAPLACE, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<5, MFA_FORM_LAPLACE, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 5 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<5, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<5, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 5 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<5, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<5, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, double>(a, budget, s);
  return cudaErrorInvalidValue;
}

cudaError_t hex_line_group_a(int n, int kind, int prec, const HexApplyArgs* items, const int64_t* first,
                                 int nitems, int64_t total, GridBudget budget, cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  if (n == 2 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return launch_line_group<2, MFA_FORM_MASS, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 2 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return launch_line_group<2, MFA_FORM_MASS, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 2 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return launch_line_group<2, MFA_FORM_LAPLACE, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 2 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return launch_line_group<2, MFA_FORM_LAPLACE, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 2 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return launch_line_group<2, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 2 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return launch_line_group<2, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 3 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return launch_line_group<3, MFA_FORM_MASS, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 3 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return launch_line_group<3, MFA_FORM_MASS, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 3 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return launch_line_group<3, MFA_FORM_LAPLACE, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 3 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return launch_line_group<3, MFA_FORM_LAPLACE, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 3 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return launch_line_group<3, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 3 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return launch_line_group<3, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 4 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return launch_line_group<4, MFA_FORM_MASS, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 4 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return launch_line_group<4, MFA_FORM_MASS, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 4 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return launch_line_group<4, MFA_FORM_LAPLACE, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 4 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return launch_line_group<4, MFA_FORM_LAPLACE, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 4 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return launch_line_group<4, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 4 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return launch_line_group<4, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 5 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return launch_line_group<5, MFA_FORM_MASS, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 5 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return launch_line_group<5, MFA_FORM_MASS, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 5 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return launch_line_group<5, MFA_FORM_LAPLACE, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 5 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return launch_line_group<5, MFA_FORM_LAPLACE, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 5 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return launch_line_group<5, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 5 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return launch_line_group<5, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  return cudaErrorInvalidValue;
}

}  // namespace mfa
