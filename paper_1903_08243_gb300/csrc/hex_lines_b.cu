// Instantiations of the line-per-thread FP32/BF16 hex action for n = 6..9
// (the other degrees live in the sibling translation unit so both compile in parallel).
#include "hex_lines.cuh"

namespace mfa {
using namespace hexl;

cudaError_t hex_line_apply_b(int n, int kind, int prec, bool f32vec, const hexl::LineArgs& a, GridBudget budget,
                                 cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  if (n == 6 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<6, MFA_FORM_MASS, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<6, MFA_FORM_MASS, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 6 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<6, MFA_FORM_MASS, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<6, MFA_FORM_MASS, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 6 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<6, MFA_FORM_LAPLACE, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<6, MFA_FORM_LAPLACE, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 6 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<6, MFA_FORM_LAPLACE, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<6, MFA_FORM_LAPLACE, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 6 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<6, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<6, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 6 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<6, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<6, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 7 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<7, MFA_FORM_MASS, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<7, MFA_FORM_MASS, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 7 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<7, MFA_FORM_MASS, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<7, MFA_FORM_MASS, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 7 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<7, MFA_FORM_LAPLACE, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<7, MFA_FORM_LAPLACE, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 7 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<7, MFA_FORM_LAPLACE, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<7, MFA_FORM_LAPLACE, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 7 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<7, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<7, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 7 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<7, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<7, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 8 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<8, MFA_FORM_MASS, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<8, MFA_FORM_MASS, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 8 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<8, MFA_FORM_MASS, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<8, MFA_FORM_MASS, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 8 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<8, MFA_FORM_LAPLACE, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<8, MFA_FORM_LAPLACE, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 8 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<8, MFA_FORM_LAPLACE, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<8, MFA_FORM_LAPLACE, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 8 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<8, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<8, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 8 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<8, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<8, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 9 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<9, MFA_FORM_MASS, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<9, MFA_FORM_MASS, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 9 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<9, MFA_FORM_MASS, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<9, MFA_FORM_MASS, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 9 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<9, MFA_FORM_LAPLACE, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<9, MFA_FORM_LAPLACE, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 9 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<9, MFA_FORM_LAPLACE, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<9, MFA_FORM_LAPLACE, MFA_PREC_BF16, double>(a, budget, s);
  if (n == 9 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return f32vec ? launch_line<9, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, float>(a, budget, s)
                  : launch_line<9, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32, double>(a, budget, s);
  if (n == 9 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return f32vec ? launch_line<9, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, float>(a, budget, s)
                  : launch_line<9, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16, double>(a, budget, s);
  return cudaErrorInvalidValue;
}

cudaError_t hex_line_group_b(int n, int kind, int prec, const HexApplyArgs* items, const int64_t* first,
                                 int nitems, int64_t total, GridBudget budget, cudaStream_t s) {
  cudaError_t e = upload_tables();
  if (e != cudaSuccess) return e;
  if (n == 6 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return launch_line_group<6, MFA_FORM_MASS, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 6 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return launch_line_group<6, MFA_FORM_MASS, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 6 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return launch_line_group<6, MFA_FORM_LAPLACE, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 6 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return launch_line_group<6, MFA_FORM_LAPLACE, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 6 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return launch_line_group<6, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 6 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return launch_line_group<6, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 7 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return launch_line_group<7, MFA_FORM_MASS, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 7 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return launch_line_group<7, MFA_FORM_MASS, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 7 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return launch_line_group<7, MFA_FORM_LAPLACE, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 7 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return launch_line_group<7, MFA_FORM_LAPLACE, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 7 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return launch_line_group<7, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 7 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return launch_line_group<7, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 8 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return launch_line_group<8, MFA_FORM_MASS, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 8 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return launch_line_group<8, MFA_FORM_MASS, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 8 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return launch_line_group<8, MFA_FORM_LAPLACE, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 8 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return launch_line_group<8, MFA_FORM_LAPLACE, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 8 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return launch_line_group<8, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 8 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return launch_line_group<8, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 9 && kind == MFA_FORM_MASS && prec == MFA_PREC_FP32)
    return launch_line_group<9, MFA_FORM_MASS, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 9 && kind == MFA_FORM_MASS && prec == MFA_PREC_BF16)
    return launch_line_group<9, MFA_FORM_MASS, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 9 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_FP32)
    return launch_line_group<9, MFA_FORM_LAPLACE, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 9 && kind == MFA_FORM_LAPLACE && prec == MFA_PREC_BF16)
    return launch_line_group<9, MFA_FORM_LAPLACE, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  if (n == 9 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_FP32)
    return launch_line_group<9, MFA_FORM_HELMHOLTZ, MFA_PREC_FP32>(items, first, nitems, total, budget, s);
  if (n == 9 && kind == MFA_FORM_HELMHOLTZ && prec == MFA_PREC_BF16)
    return launch_line_group<9, MFA_FORM_HELMHOLTZ, MFA_PREC_BF16>(items, first, nitems, total, budget, s);
  return cudaErrorInvalidValue;
}

}  // namespace mfa
